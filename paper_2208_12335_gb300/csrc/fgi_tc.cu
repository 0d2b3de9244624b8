// Tensor-core path for sm_103a: basis evaluation into swizzled BF16 operand
// images, the H contraction h_b = Phi_b^T diag(w v) Phi_b on tcgen05 (or
// s Psi_b^T Psi_b with Psi = Phi sqrt|w v| where w v has one sign s) with a
// fixed-point scatter into H, the D_b gather, and the density contraction
// n_p = sum_j (D_b Phi_b^T)_jp phi_j(p) on tcgen05.
//
// Precision: every value x entering a contraction is split into three BF16
// terms x = x0 + x1 + x2: x0 a fixed-point digit on a power-of-two grid per
// row (H) or per point (density), chosen so that every partial sum of
// x0*y0 products is exact in FP32, and x1, x2 the BF16 split of the
// remainder.  H and the density accumulate the 8 products of combined
// order <= 3 except x2*y2; x0*y0 has its own FP32
// accumulator in tensor memory, the others a second one.  Cross-batch sums:
// H in 2^-40 fixed point (int64 atomics, deterministic), the density in
// FP64.  n_split = 1 keeps x0*y0 only (plain BF16).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/fgi.h"
#include "fgi_basis.cuh"
#include "fgi_dd.cuh"
#include "fgi_index.cuh"
#include "fgi_tc.h"

namespace fgi {

namespace {

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s: a wait that long means a bug

// Bounded wait on an mbarrier phase (time-out: kStatusTimeout), with a CTA-wide abort flag: once any wait of the CTA has
// timed out, every later wait fails at once, so that the roles finish their
// loops quickly with unchanged control flow (no named barrier is skipped).
__device__ __forceinline__ bool mbar_wait_a(uint64_t *bar, uint32_t parity, int *status, volatile int *abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (global_ns() - t0 > kWaitLimitNs) {
            *abort = 1;
            atomicOr(status, kStatusTimeout);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns: thread (lane) gets its row's 32 values
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, 128-byte swizzle (tcgen05 format: version 1).
// K-major: rows of 64 BF16 (128 B), 8-row atoms of 1 KB; sbo = atom stride.
// MN-major: lbo = stride between 64-element MN atoms, sbo = stride between
// 8-row K groups.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: kind::f16, BF16 x BF16 -> F32, dense.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// --------------------------------------------------------------- splitting
__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// byte offset of the 16-byte unit (row r, 8-column group g) inside chunk (blk, c)
__device__ __forceinline__ long long unit_offset(int blk, int nchunk, int c, int r, int g)
{
    return ((long long)(blk * nchunk + c) * 16 + (r >> 3)) * 1024 + (r & 7) * 128 + ((g ^ (r & 7)) << 4);
}

// Normalisation constants of the real spherical harmonics as double-floats.
#define FGI_DF_CONST(c) {(float)(c), (float)((c) - (double)(float)(c))}
__constant__ float2 kYlmC[10] = {
    FGI_DF_CONST(0.28209479177387814),  // l0
    FGI_DF_CONST(0.4886025119029199),   // l1
    FGI_DF_CONST(1.0925484305920792),   // l2: xy, yz, xz
    FGI_DF_CONST(0.31539156525252005),  // l2: 2z^2 - x^2 - y^2
    FGI_DF_CONST(0.5462742152960396),   // l2: x^2 - y^2
    FGI_DF_CONST(0.5900435899266435),   // l3: y(3x^2 - y^2), x(x^2 - 3y^2)
    FGI_DF_CONST(2.890611442640554),    // l3: xyz
    FGI_DF_CONST(0.4570457994644658),   // l3: y(4z^2 - x^2 - y^2), x(...)
    FGI_DF_CONST(0.3731763325901154),   // l3: z(2z^2 - 3x^2 - 3y^2)
    FGI_DF_CONST(1.445305721320277)};   // l3: z(x^2 - y^2)
#undef FGI_DF_CONST

// r^l Y_lm = C_lm * Q_lm(x, y, z): Q with small integer coefficients (FP32),
// the constant index into kYlmC.
__device__ __forceinline__ void ylm_poly_f32(int l, float x, float y, float z, float *Q, int *ci)
{
    if (l == 0) {
        Q[0] = 1.f; ci[0] = 0;
    } else if (l == 1) {
        Q[0] = y; Q[1] = z; Q[2] = x;
        ci[0] = ci[1] = ci[2] = 1;
    } else if (l == 2) {
        Q[0] = x * y; Q[1] = y * z; Q[2] = 2.f * z * z - x * x - y * y; Q[3] = x * z; Q[4] = x * x - y * y;
        ci[0] = 2; ci[1] = 2; ci[2] = 3; ci[3] = 2; ci[4] = 4;
    } else {
        const float q = 4.f * z * z - x * x - y * y;
        Q[0] = y * (3.f * x * x - y * y); Q[1] = x * y * z; Q[2] = y * q;
        Q[3] = z * (2.f * z * z - 3.f * x * x - 3.f * y * y); Q[4] = x * q; Q[5] = z * (x * x - y * y);
        Q[6] = x * (x * x - 3.f * y * y);
        ci[0] = 5; ci[1] = 6; ci[2] = 7; ci[3] = 8; ci[4] = 7; ci[5] = 9; ci[6] = 5;
    }
}

// 3-term BF16 split of a double-float value
__device__ __forceinline__ void split3_df(df x, __nv_bfloat16 &a, __nv_bfloat16 &b, __nv_bfloat16 &c)
{
    a = __float2bfloat16_rn(x.hi);
    float r = (x.hi - __bfloat162float(a)) + x.lo;
    b = __float2bfloat16_rn(r);
    r -= __bfloat162float(b);
    c = __float2bfloat16_rn(r);
}

__device__ __forceinline__ void store_split8_df(uint8_t *dst, long long plane, const df *x, int n_split)
{
    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        __nv_bfloat16 a0, a1, a2, b0, b1, b2;
        split3_df(x[2 * q], a0, a1, a2);
        split3_df(x[2 * q + 1], b0, b1, b2);
        w0[q] = pack_bf16(a0, b0);
        w1[q] = pack_bf16(a1, b1);
        w2[q] = pack_bf16(a2, b2);
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    if (n_split > 1) *reinterpret_cast<uint4 *>(dst + plane) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    if (n_split > 2) *reinterpret_cast<uint4 *>(dst + 2 * plane) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
}

// Split with a fixed-point leading term: x0 = m * unit, m = rint(x / unit),
// unit = 2^(e-7) with 2^e >= the row's largest |x|, so |m| <= 128 and every
// product x0*y0 of a row pair is an integer multiple of unit_x*unit_y not
// exceeding 2^14 in units; a sum of up to 1024 of them (a batch) is exact in
// FP32 whatever the accumulator's rounding.  The remainder x - x0 is split
// relative to itself into two BF16 terms.
__device__ __forceinline__ void split_fixed(df x, float scale, float unit, __nv_bfloat16 &a,
                                            __nv_bfloat16 &b, __nv_bfloat16 &c)
{
    const float x0 = rintf(x.hi * scale) * unit;
    // x.hi - x0 is exact: x0 is a multiple of unit, and unit >= ulp(x.hi)
    // because |x.hi| <= 2^e (1 + 2^-12) and unit = 2^(e - bits), bits <= 8
    const float d = x.hi - x0;
    a = __float2bfloat16_rn(x0);
    b = __float2bfloat16_rn(d);
    c = __float2bfloat16_rn((d - __bfloat162float(b)) + x.lo);
}

__device__ __forceinline__ void store_fixed8(uint8_t *dst, long long plane, const df *x, float scale, float unit)
{
    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        __nv_bfloat16 a0, a1, a2, b0, b1, b2;
        split_fixed(x[2 * q], scale, unit, a0, a1, a2);
        split_fixed(x[2 * q + 1], scale, unit, b0, b1, b2);
        w0[q] = pack_bf16(a0, b0);
        w1[q] = pack_bf16(a1, b1);
        w2[q] = pack_bf16(a2, b2);
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    *reinterpret_cast<uint4 *>(dst + plane) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *reinterpret_cast<uint4 *>(dst + 2 * plane) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
}

// Power-of-two scale 2^(b-e) and unit 2^(e-b) for a row whose largest |x|
// is mx: |x| * scale <= 2^b.  b digit bits keep the exact sum: 2^(2b) times
// the contraction depth must not exceed 2^24.  Rows below 1e-30 (negligible
// against any stored value) put everything in the remainder terms.
__device__ __forceinline__ int fixed_bits(int depth)
{
    int b = 7;
    while (b > 1 && ((long long)depth << (2 * b)) > (1ll << 24)) b--;
    return b;
}

// Leading-digit width: 8 bits when the row's sum S = sum|x|/2^e <= 200 (then
// every row-pair sum stays below 65536 S + 128 K < 2^24 for K <= 8192),
// otherwise the width that keeps depth x 2^(2b) <= 2^24.
__device__ __forceinline__ void fixed_scale_adaptive(float mx, float sum, int depth, float &scale, float &unit)
{
    if (!(mx > 1e-30f)) {
        scale = 0.f;
        unit = 0.f;
        return;
    }
    int e;
    frexpf(mx * (1.f + 1.f / 4096.f), &e);
    const float S = ldexpf(sum, -e) * 1.001f;
    const int bits = (S <= 200.f) ? 8 : fixed_bits(depth);
    scale = ldexpf(1.f, bits - e);
    unit = ldexpf(1.f, e - bits);
}


// FP32 u(d)/d^(l+1) for the first passes, which only take maxima and sums
// of |phi| from it (a relative error of a few ulp is far inside the 2^-12
// margin of the fixed-point grids); inv_d = 1/d, computed once per point.
// tab: the radial's interval-0 entry (hi coefficients), entries `step` float4 apart.
__device__ __forceinline__ float radial_over_d_f32(const DevRadial &R, const float4 *tab, int step, float d,
                                                   float inv_d)
{
    if (d >= R.rcut_f) return 0.f;
    if (d < 1e-12f) return R.l == 0 ? __ldg(tab).y * R.inv_h_hi : 0.f;
    const float s = d * R.inv_h_hi;
    int k = (int)s;
    if (k > R.nk - 2) k = R.nk - 2;
    const float t = s - (float)k;
    const float4 c = __ldg(tab + (long long)k * step);
    const float u = c.x + t * (c.y + t * (c.z + t * c.w));
    const float i2 = inv_d * inv_d;
    const float ip = R.l == 0 ? inv_d : (R.l == 1 ? i2 : (R.l == 2 ? i2 * inv_d : i2 * i2));
    return u * ip;
}

constexpr int kPhiValStride = 33;   // float2 per row of phi_smem (32 points + padding)

// Interval-0 entry of shell sh's spline and the distance between interval
// entries: the species' interleaved table when its shells share one grid.
__device__ __forceinline__ const float4 *spline_tab(const DevPlan &P, const DevSpecies &S, const DevRadial &R, int sh,
                                                    int &step)
{
    if (S.shared_grid) {
        step = 2 * S.n_shell;
        return P.scoef + S.scoef_off + 2 * sh;
    }
    step = 2;
    return P.coef_dd + 2 * R.coef_off;
}

// ----------------------------------------- lane-per-point basis evaluation
// One lane evaluates every function of one atom at its own point and hands
// each value straight to an emitter (split + 16-bit stores into the operand
// image): values never pass through shared memory, and the 32 lanes of a
// warp (32 consecutive points, one atom) store 64 contiguous bytes of one
// image row per plane.  The geometry (offset, distance, 1/d^(l+1)) is
// double-float once per (point, atom); the radial factor once per shell,
// times the per-point scale of each image; the angular polynomial FP32.
// (Two points per lane with 32-bit stores of BF16 pairs was measured
// slower: the doubled per-lane state costs occupancy or spills, and these
// kernels wait mostly on their loads.)

// byte offset of element (row r, point p) in the image chunk grid of block I
// (below 2^31: a batch's image plane is at most 64 blocks x 16 chunks x 16 KB)
__device__ __forceinline__ int elem_offset(int I, int nc_alloc, int r, int p)
{
    const int g = (p >> 3) & 7;
    return ((I * nc_alloc + (p >> 6)) * 16 + (r >> 3)) * 1024 + (r & 7) * 128 + ((g ^ (r & 7)) << 4) + (p & 7) * 2;
}

// One value split on its row's or point's grid (split_fixed; NSPLIT 1:
// plain BF16) and stored as one 16-bit BF16 per plane
template <int NSPLIT>
__device__ __forceinline__ void store_value(uint8_t *dst, long long plane, df x, float scale, float unit)
{
    if (NSPLIT == 3) {
        __nv_bfloat16 a, b, c;
        split_fixed(x, scale, unit, a, b, c);
        *reinterpret_cast<unsigned short *>(dst) = __bfloat16_as_ushort(a);
        *reinterpret_cast<unsigned short *>(dst + plane) = __bfloat16_as_ushort(b);
        *reinterpret_cast<unsigned short *>(dst + 2 * plane) = __bfloat16_as_ushort(c);
    } else {
        *reinterpret_cast<unsigned short *>(dst) = __bfloat16_as_ushort(__float2bfloat16_rn(x.hi));
    }
}

__device__ __forceinline__ void store_zero(uint8_t *dst, long long plane, int nsplit)
{
    *reinterpret_cast<unsigned short *>(dst) = 0;
    if (nsplit > 1) {
        *reinterpret_cast<unsigned short *>(dst + plane) = 0;
        *reinterpret_cast<unsigned short *>(dst + 2 * plane) = 0;
    }
}

// Ratios of the other normalisation constants of an l shell to its first
// (the spline tables of the lane kernels hold u times the first constant):
// l = 2: C(2z^2-x^2-y^2)/C(xy) = 1/(2 sqrt 3); l = 3: C(z(x^2-y^2))/C(y(3x^2-y^2))
// = sqrt 6 (C(xyz) is twice that), sqrt(3/5) and sqrt(2/5).
#define FGI_DF_CONST(c) {(float)(c), (float)((c) - (double)(float)(c))}
__constant__ float2 kYlmRatio[4] = {
    FGI_DF_CONST(0.28867513459481287),   // 1/(2 sqrt 3)
    FGI_DF_CONST(2.449489742783178),     // sqrt 6
    FGI_DF_CONST(0.7745966692414834),    // sqrt(3/5)
    FGI_DF_CONST(0.6324555320336759)};   // sqrt(2/5)
#undef FGI_DF_CONST

// r^l Y_lm / C_l (C_l the first constant of the shell) = K_g * Q_m: Q in
// FP32 with the exact factors 2 and 1/2 folded in, g the index of the
// ratio K (0: K = 1).
template <int L>
__device__ __forceinline__ void ylm_poly_unit(float x, float y, float z, float *Q, int *g)
{
    if (L == 0) {
        Q[0] = 1.f; g[0] = 0;
    } else if (L == 1) {
        Q[0] = y; Q[1] = z; Q[2] = x;
        g[0] = g[1] = g[2] = 0;
    } else if (L == 2) {
        Q[0] = x * y; Q[1] = y * z; Q[2] = 2.f * z * z - x * x - y * y; Q[3] = x * z;
        Q[4] = 0.5f * (x * x - y * y);
        g[0] = 0; g[1] = 0; g[2] = 1; g[3] = 0; g[4] = 0;
    } else {
        const float q = 4.f * z * z - x * x - y * y;
        Q[0] = y * (3.f * x * x - y * y); Q[1] = 2.f * (x * y * z); Q[2] = y * q;
        Q[3] = z * (2.f * z * z - 3.f * x * x - 3.f * y * y); Q[4] = x * q; Q[5] = z * (x * x - y * y);
        Q[6] = x * (x * x - 3.f * y * y);
        g[0] = 0; g[1] = 1; g[2] = 2; g[3] = 3; g[4] = 2; g[5] = 1; g[6] = 0;
    }
}

// the 2l+1 values of one shell for NIMG radial factors rk[k] (= C_l
// u/d^(l+1) times the image's per-point scale), handed to the emitter as
// unnormalised double-floats (the split uses hi + lo only)
template <int L, int NIMG, class Emit>
__device__ __forceinline__ void emit_shell_lane(const df *rk, float x, float y, float z, int f0, int f_lo, int f_hi,
                                                Emit &emit)
{
    constexpr int NM = 2 * L + 1;
    constexpr int NG = L < 2 ? 1 : (L == 2 ? 2 : 4);
    constexpr int G0 = L == 2 ? 0 : 1;               // first kYlmRatio entry of groups 1..
    float Q[NM];
    int gi[7];
    ylm_poly_unit<L>(x, y, z, Q, gi);
    df rc[NIMG][NG];
#pragma unroll
    for (int k = 0; k < NIMG; k++) {
        rc[k][0] = rk[k];
#pragma unroll
        for (int c = 1; c < NG; c++)
            rc[k][c] = df_mul(rk[k], df{kYlmRatio[G0 + c - 1].x, kYlmRatio[G0 + c - 1].y});
    }
    const bool whole = f0 >= f_lo && f0 + NM <= f_hi;
#pragma unroll
    for (int m = 0; m < NM; m++) {
        const int fm = f0 + m;
        if (!whole && (fm < f_lo || fm >= f_hi)) continue;
        df val[NIMG];
#pragma unroll
        for (int k = 0; k < NIMG; k++) val[k] = df_mul_f_raw(rc[k][gi[m]], Q[m]);
        emit(fm, val);
    }
}

// Every function [f_lo, f_hi) of atom `atom` (species S, shell table sh_tab
// indexed from S.shell0) at the point whose double-float coordinates pp
// holds (nullptr: no point).  emit(f, val[NIMG]) receives phi times the
// image's scale (SCALED false: image 0 unscaled); emit0(f) a value that is
// zero in every image (beyond the species' cutoff, or no point); zero_all()
// is called by all 32 lanes of the warp, instead of emit0, when every lane
// is beyond the cutoff or has no point (the warp's part of the image is then
// cleared with 16-byte stores).  The per-point scales are folded into the
// powers 1/d^(l+1) once per (point, atom).  All 32 lanes of the warp call
// this together, for the same atom.
template <int NIMG, bool SCALED, class Emit, class Emit0, class Zero>
__device__ __forceinline__ void eval_atom_lane(const DevPlan &P, const DevSpecies &S, const DevShell *sh_tab,
                                               int atom, const float *pp, int f_lo, int f_hi, const df *scale,
                                               Emit &emit, Emit0 &emit0, Zero &zero_all)
{
    const df zero{0.f, 0.f};
    bool none = pp == nullptr;
    const float *aa = P.atom_dd + 6 * atom;
    if (!none) {
        // beyond the species' largest cutoff every value is zero (FP32
        // distance, relative error ~1e-7, against the cutoff with a 1e-5 margin)
        const float xf = (pp[0] - aa[0]) + (pp[1] - aa[1]);
        const float yf = (pp[2] - aa[2]) + (pp[3] - aa[3]);
        const float zf = (pp[4] - aa[4]) + (pp[5] - aa[5]);
        const float rcs = (float)S.rcut * 1.00001f;
        none = xf * xf + yf * yf + zf * zf > rcs * rcs;
    }
    if (__all_sync(0xffffffffu, none)) {
        zero_all();
        return;
    }
    if (none) {
        for (int f = f_lo; f < f_hi; f++) emit0(f);
        return;
    }
    // offset from the atom (the rounding of the low parts differs from point
    // to point), d^2 (terms of one sign), 1/d from a refined rsqrtf, d = d^2/d
    const df x = df_sub_sloppy(df{pp[0], pp[1]}, df{aa[0], aa[1]});
    const df y = df_sub_sloppy(df{pp[2], pp[3]}, df{aa[2], aa[3]});
    const df z = df_sub_sloppy(df{pp[4], pp[5]}, df{aa[4], aa[5]});
    const df d2 = df_add_sloppy(df_add_sloppy(df_mul(x, x), df_mul(y, y)), df_mul(z, z));
    const bool origin = d2.hi < 1e-24f;                 // d < 1e-12
    df d = zero, i0 = zero;
    if (!origin) {
        i0 = df_rsqrt(d2);
        d = df_mul(d2, i0);
    }
    // 1/d^(l+1) for l <= lmax, times each image's scale
    df ip[NIMG][4];
    {
        df pw[4];
        pw[0] = i0;
        pw[1] = S.lmax >= 1 ? df_mul(i0, i0) : zero;
        pw[2] = S.lmax >= 2 ? df_mul(pw[1], i0) : zero;
        pw[3] = S.lmax >= 3 ? df_mul(pw[2], i0) : zero;
#pragma unroll
        for (int k = 0; k < NIMG; k++) {
            const bool sc = SCALED || k > 0;
#pragma unroll
            for (int q = 0; q < 4; q++) ip[k][q] = (sc && q <= S.lmax) ? df_mul(pw[q], scale[k]) : pw[q];
        }
    }
    float grid_hi = -1.f, grid_lo = 0.f, t = 0.f, tl = 0.f;
    int grid_nk = -1, kk = 0;
    const float4 *sc = nullptr;
    if (S.shared_grid && !origin) {
        const df sd = df_mul(d, df{S.inv_h_hi, S.inv_h_lo});
        kk = (int)floorf(sd.hi);
        kk = max(0, min(kk, S.nk - 2));
        t = sd.hi - (float)kk;
        tl = sd.lo;
        sc = P.scoefn + S.scoef_off + 2 * ((long long)kk * S.n_shell);
    }
    // the shells grouped by l: the power 1/d^(l+1) and the angular
    // polynomial's form are fixed within a group
    int sh = 0;
    auto shells_of_l = [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        constexpr int NM = 2 * L + 1;
        const int end = sh + S.nl[L];
        for (; sh < end; sh++) {
            const DevShell R = sh_tab[S.shell0 + sh];
            const int f = R.fn0;
            if (f + NM <= f_lo || f >= f_hi) continue;
            df uu = zero;                               // C_l u(d), or its limit C_0 u'(0) d at the origin
            bool live = d.hi < R.rcut_f;
            if (live) {
                if (origin) {
                    live = L == 0;
                    if (live) {
                        const float4 ch = __ldg(P.coef_ddn + 2 * R.coef_off), cl = __ldg(P.coef_ddn + 2 * R.coef_off + 1);
                        uu = df_mul(df{ch.y, cl.y}, df{R.inv_h_hi, R.inv_h_lo});   // the l = 0 limit C_0 c1/h
                    }
                } else {
                    const float4 *ce;
                    if (sc) {
                        ce = sc + 2 * sh;
                    } else {
                        if (R.inv_h_hi != grid_hi || R.inv_h_lo != grid_lo || R.nk != grid_nk) {
                            grid_hi = R.inv_h_hi;
                            grid_lo = R.inv_h_lo;
                            grid_nk = R.nk;
                            const df s2 = df_mul(d, df{R.inv_h_hi, R.inv_h_lo});
                            kk = (int)floorf(s2.hi);
                            kk = max(0, min(kk, R.nk - 2));
                            t = s2.hi - (float)kk;
                            tl = s2.lo;
                        }
                        ce = P.coef_ddn + 2 * (R.coef_off + kk);
                    }
                    // u = c0 + t c1 + t^2 (c2 + t c3): c0 + t c1 in double-float
                    const float4 ch = __ldg(ce);
                    const float4 cl = __ldg(ce + 1);
                    const df lin = df_two_prod(t, ch.y);
                    const float lin_lo = fmaf(t, cl.y, fmaf(tl, ch.y, lin.lo));
                    const float quad = (t * t) * fmaf(t, ch.w, ch.z);
                    uu = df_two_sum(ch.x, lin.hi);
                    uu = df_two_sum(uu.hi, uu.lo + ((cl.x + lin_lo) + quad));
                }
            }
            if (!live) {
                const int m0 = max(f, f_lo), m1 = min(f + NM, f_hi);
                for (int m = m0; m < m1; m++) emit0(m);
                continue;
            }
            df rk[NIMG];
#pragma unroll
            for (int k = 0; k < NIMG; k++)
                rk[k] = origin ? ((SCALED || k > 0) ? df_mul(uu, scale[k]) : uu) : df_mul(uu, ip[k][L]);
            emit_shell_lane<L, NIMG>(rk, x.hi, y.hi, z.hi, f, f_lo, f_hi, emit);
        }
    };
    shells_of_l(std::integral_constant<int, 0>{});
    if (S.lmax >= 1) shells_of_l(std::integral_constant<int, 1>{});
    if (S.lmax >= 2) shells_of_l(std::integral_constant<int, 2>{});
    if (S.lmax >= 3) shells_of_l(std::integral_constant<int, 3>{});
}

// the species' shells for one CTA: shared memory when they fit
constexpr int kMaxShellsSmem = 64;
__device__ __forceinline__ const DevShell *stage_shells(const DevPlan &P, DevShell *smem)
{
    if (P.n_shells > kMaxShellsSmem) return P.shells;
    for (int i = threadIdx.x; i < P.n_shells; i += blockDim.x) smem[i] = P.shells[i];
    return smem;                                    // valid after the caller's next __syncthreads
}

// H images of one 128-row block: warp tasks (atom of the block, 32-point
// group), lane = point.  NIMG 1: psi = phi sqrt|w v| on the second grid set;
// NIMG 2: phi (first set) and w v phi (second set) into two images.
template <int NIMG, int NSPLIT>
__device__ __forceinline__ void h_image_lanes(const DevPlan &P, const DevBatch &B, const TcBatch &T,
                                              const DevAct *act, const DevShell *sh_tab, int I, int e0, int ne,
                                              uint8_t *img0, uint8_t *img1, const float2 *wvs,
                                              const float (*fsc)[128][2])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int r0 = I * 128;
    const int ng = 2 * T.nc;                       // 32-point groups covering the image's chunks
    for (int task = warp; task < ne * ng; task += nwarp) {
        const int eq = task / ng, q = task - eq * ng;
        const DevAct A = act[e0 + eq];
        const DevSpecies S = P.species[P.atom_species[A.atom]];
        const int f_lo = max(0, r0 - A.fn_loc), f_hi = min(S.n_fn, r0 + 128 - A.fn_loc);
        const int p = q * 32 + lane;
        const bool live = p < B.np;
        const float *pp = live ? P.pts_dd + 6 * (B.pt0 + p) : nullptr;
        df scale[NIMG];
        const float2 s2 = live ? wvs[p] : make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < NIMG; k++) scale[k] = df{s2.x, s2.y};
        const int rb = A.fn_loc - r0;
        auto emit = [&](int f, const df *val) {
            const int r = rb + f;
            const int off = elem_offset(I, T.nc_alloc, r, p);
#pragma unroll
            for (int k = 0; k < NIMG; k++) {
                const int set = NIMG == 1 ? 1 : k;
                store_value<NSPLIT>((k == 0 ? img0 : img1) + off, T.plane_phi, val[k], fsc[set][r][0],
                                    fsc[set][r][1]);
            }
        };
        auto emit0 = [&](int f) {
            const int off = elem_offset(I, T.nc_alloc, rb + f, p);
#pragma unroll
            for (int k = 0; k < NIMG; k++) store_zero((k == 0 ? img0 : img1) + off, T.plane_phi, NSPLIT);
        };
        // the warp's 32 columns of rows rb + [f_lo, f_hi): four 16-byte units
        // per row and plane
        auto zero_all = [&]() {
            const int pc = q * 32;
            for (int u = lane; u < (f_hi - f_lo) * 4; u += 32) {
                const int off = elem_offset(I, T.nc_alloc, rb + f_lo + (u >> 2), pc + (u & 3) * 8);
#pragma unroll
                for (int k = 0; k < NIMG; k++)
#pragma unroll
                    for (int pl = 0; pl < NSPLIT; pl++)
                        *reinterpret_cast<uint4 *>((k == 0 ? img0 : img1) + off + pl * T.plane_phi) =
                            make_uint4(0u, 0u, 0u, 0u);
            }
        };
        eval_atom_lane<NIMG, NIMG == 1>(P, S, sh_tab, A.atom, pp, f_lo, f_hi, scale, emit, emit0, zero_all);
    }
}

// -------------------------------------------- basis -> operand images (K1)
// CTA per (batch, 128-row block).  A first FP32 pass takes the rows' maxima
// and sums for the fixed-point grids; then, for each 32-point half chunk,
// phi of the block's rows is evaluated into shared memory and the split
// planes of psi = phi sqrt|w v| (batches where w v has one sign) or of phi
// and w v phi (mixed signs) are written as swizzled 16-byte units.
//
// The radial factor N_lm u(d)/d^(l+1) -- shared by all angular points of a
// radial shell, so its rounding would be systematic -- is evaluated in
// double-float from a double-float spline table and double-float
// coordinates; only the angular polynomial Q_lm(x, y, z) is FP32 (its
// rounding varies from point to point).

constexpr int kPhiThreads = 256;
constexpr int kDistCacheFloats = 128 * kPhiValStride * 2;     // the dynamic buffer, as floats

// FP32 distance from atom `atom` to point `pt` (from the double-float
// coordinates), for the bounds of the digit grids
__device__ __forceinline__ float point_atom_dist_f32(const DevPlan &P, int atom, long long pt)
{
    const float *aa = P.atom_dd + 6 * atom;
    const float *pp = P.pts_dd + 6 * pt;
    const float x = (pp[0] - aa[0]) + (pp[1] - aa[1]);
    const float y = (pp[2] - aa[2]) + (pp[3] - aa[3]);
    const float z = (pp[4] - aa[4]) + (pp[5] - aa[5]);
    return sqrtf(x * x + y * y + z * z);
}

__global__ void __launch_bounds__(kPhiThreads, 4) k_tc_phi(DevPlan P, const TcBatch *tb, const WorkItem *items,
                                                uint8_t *ws, const double *v, int n_split, int fixed,
                                                int *bsign, int bound)
{
    extern __shared__ float2 phi_smem[];             // [128][kPhiValStride] double-float values
    __shared__ float2 wvs[kMaxBatchPoints];         // per-point image scale (double-float)
    __shared__ DevShell shs[kMaxShellsSmem];
    __shared__ unsigned int rowmax[2][128];          // |phi|, |w v phi| maxima (float bits)
    __shared__ float rowsum[2][128];                 // sums of |phi|, |w v phi| over the points
    __shared__ float fsc[2][128][2];                 // per row: scale, unit
    __shared__ float wvf[kMaxBatchPoints];           // |w v| per point (FP32), first pass
    const WorkItem it = items[blockIdx.x];
    const DevBatch B = P.batches[it.batch];
    const TcBatch T = tb[it.batch];
    const int I = it.ti;
    const int r0 = I * 128;
    const DevAct *act = P.act + B.act0;
    const int rend = min(r0 + 128, B.nfn);
    const int e0 = find_act(act, B.n_act, r0);
    const int e1 = find_act(act, B.n_act, rend - 1);
    const int ne = e1 - e0 + 1;
    uint8_t *phi_img = ws + T.img_phi;
    uint8_t *a_img = ws + T.img_aux;
    // the species' shells (visible after the barrier below)
    const DevShell *sh_tab = stage_shells(P, shs);
    // sign of w v over the batch: one sign s (or zero) everywhere lets H use a
    // single image psi = phi sqrt|w v| for both operands, H = s psi^T psi;
    // mixed signs keep the phi and w v phi images
    bool pos = false, neg = false;
    for (int p = threadIdx.x; p < B.np; p += blockDim.x) {
        const double wv = P.pw[B.pt0 + p] * v[B.pt0 + p];
        pos |= wv > 0.0;
        neg |= wv < 0.0;
    }
    pos = __syncthreads_or(pos) != 0;
    neg = __syncthreads_or(neg) != 0;
    const int sgn = (pos && neg) ? 0 : (neg ? -1 : 1);
    if (I == 0 && threadIdx.x == 0) bsign[it.batch] = sgn;
    if (fixed && bound) {
        // row bounds from the tables: per (atom, shell) and point one lookup
        // of the suffix bound of |u(r)/r| at the point's distance (knot index
        // taken from below), times sqrt|w v| (psi) or |w v| (w v phi) of the
        // point; the maximum over the points times max |Y_lm| bounds each
        // row, and the same products summed over the points bound the row
        // sums, so that rows whose sum allows it keep an 8-bit digit.
        for (int q = threadIdx.x; q < 256; q += blockDim.x) {
            (&rowmax[0][0])[q] = 0u;          // rows past n_b stay zero
            (&rowsum[0][0])[q] = 0.f;
        }
        for (int p = threadIdx.x; p < B.np; p += blockDim.x) {
            const float a = fabsf((float)(P.pw[B.pt0 + p] * v[B.pt0 + p])) * (1.f + 1.f / 1048576.f);
            wvf[p] = fminf(sgn != 0 ? sqrtf(a) * (1.f + 1.f / 1048576.f) : a, 1.0e30f);
        }
        // distances of the block's atoms to the batch's points (FP32), once,
        // in the dynamic buffer when they fit
        float *dcache = reinterpret_cast<float *>(phi_smem);
        const bool dcached = ne * B.np <= kDistCacheFloats;
        if (dcached) {
            for (int q = threadIdx.x; q < ne * B.np; q += blockDim.x) {
                const int eq = q / B.np, p = q - eq * B.np;
                dcache[q] = point_atom_dist_f32(P, act[e0 + eq].atom, B.pt0 + p);
            }
        }
        __syncthreads();
        // warp tasks (atom of the block, shell): the lanes stride over the
        // batch's points, one lookup per point, and keep the maxima and sums in
        // registers; one warp reduction per task, whose rows it alone writes
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
        int job0 = 0;
        for (int e = e0; e <= e1; e++) {
            const DevAct A = act[e];
            const DevSpecies S = P.species[P.atom_species[A.atom]];
            const int f_lo = max(0, r0 - A.fn_loc), f_hi = min(S.n_fn, r0 + 128 - A.fn_loc);
            const int first = ((warp - job0) % nwarp + nwarp) % nwarp;
            job0 += S.n_shell;
            for (int sh = first; sh < S.n_shell; sh += nwarp) {
                const DevShell R = sh_tab[S.shell0 + sh];
                const int nm = 2 * R.l + 1, f1 = R.fn0;
                if (f1 + nm <= f_lo || f1 >= f_hi) continue;
                const float rcl = R.rcut_f * 1.00001f;
                const float *bt = P.rbound + R.bound_off;
                float m0 = 0.f, m1 = 0.f, s0 = 0.f, s1 = 0.f;
                for (int p = lane; p < B.np; p += 32) {
                    const float d = dcached ? dcache[(e - e0) * B.np + p] : point_atom_dist_f32(P, A.atom, B.pt0 + p);
                    if (d < rcl) {
                        // knot index taken from below against FP32 rounding of d
                        const int ki = min(max((int)(d * 0.999999f * R.inv_h_hi), 0), R.nk - 2);
                        const float t = __ldg(bt + ki);
                        const float tw = t * wvf[p];
                        m0 = fmaxf(m0, t);
                        m1 = fmaxf(m1, tw);
                        s0 += t;
                        s1 += tw;
                    }
                }
                m0 = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m0)));
                m1 = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m1)));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                }
                // lane m folds function m of the shell into its row
                const int fr = f1 + lane;
                if (lane < nm && m0 > 0.f && fr >= f_lo && fr < f_hi) {
                    const int row = A.fn_loc + fr - r0;
                    const float yl = __ldg(P.rbound + R.l * R.l + lane);
                    rowmax[0][row] = __float_as_uint(fminf(m0 * yl, 1.0e30f));
                    rowmax[1][row] = __float_as_uint(fminf(m1 * yl, 1.0e30f));
                    rowsum[0][row] = fminf(s0 * 1.0001f * yl, 1.0e30f);   // 1.0001: FP32 sums
                    rowsum[1][row] = fminf(s1 * 1.0001f * yl, 1.0e30f);
                }
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < 256; q += blockDim.x) {
            const int which = q >> 7, r = q & 127;
            float sc, un;
            fixed_scale_adaptive(__uint_as_float(rowmax[which][r]), rowsum[which][r], T.nc * 64, sc, un);
            fsc[which][r][0] = sc;
            fsc[which][r][1] = un;
        }
        __syncthreads();
    } else if (fixed) {
        // pass 1: row maxima and sums of |phi| and |w v phi| (or of |psi|,
        // kept in the second set) over the batch's points (FP32).  One warp
        // per (atom, shell) of the block; lanes stride over the points and
        // keep per-function partials in registers.
        for (int q = threadIdx.x; q < 256; q += blockDim.x) {
            (&rowmax[0][0])[q] = 0u;          // rows past n_b stay zero
            (&rowsum[0][0])[q] = 0.f;
        }
        for (int p = threadIdx.x; p < B.np; p += blockDim.x) {
            const float a = fabsf((float)(P.pw[B.pt0 + p] * v[B.pt0 + p]));
            wvf[p] = fminf(sgn != 0 ? sqrtf(a) : a, 1.0e30f);
        }
        // FP32 offsets and distances of the block's atoms to the batch's points,
        // once, in the (not yet used) value buffer when they fit: every shell
        // job of an atom reads them instead of recomputing them
        float4 *geo = reinterpret_cast<float4 *>(phi_smem);
        const bool geo_cached = ne * B.np <= 128 * kPhiValStride / 2;    // float4 slots of the buffer
        if (geo_cached) {
            for (int q = threadIdx.x; q < ne * B.np; q += blockDim.x) {
                const int eq = q / B.np, p = q - eq * B.np;
                const float *aa = P.atom_dd + 6 * act[e0 + eq].atom;
                const float *pp = P.pts_dd + 6 * (B.pt0 + p);
                const float x = (pp[0] + pp[1]) - (aa[0] + aa[1]);
                const float y = (pp[2] + pp[3]) - (aa[2] + aa[3]);
                const float z = (pp[4] + pp[5]) - (aa[4] + aa[5]);
                geo[q] = make_float4(x, y, z, sqrtf(x * x + y * y + z * z));
            }
        }
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
        int job = 0;
        for (int e = e0; e <= e1; e++) {
            const DevAct A = act[e];
            const DevSpecies S = P.species[P.atom_species[A.atom]];
            const int f_lo = max(0, r0 - A.fn_loc), f_hi = min(S.n_fn, r0 + 128 - A.fn_loc);
            const float *aa = P.atom_dd + 6 * A.atom;
            const float ax = aa[0] + aa[1], ay = aa[2] + aa[3], az = aa[4] + aa[5];
            int f = 0;
            for (int sh = 0; sh < S.n_shell; sh++) {
                const DevRadial R = P.radials[P.shell_rad[S.shell0 + sh]];
                const int nm = 2 * R.l + 1;
                const int f1 = f;
                f += nm;
                if (f <= f_lo || f1 >= f_hi) continue;
                if ((job++ % nwarp) != warp) continue;
                int tstep;
                const float4 *tab = spline_tab(P, S, R, sh, tstep);
                float mx[7], sm[7], mxw[7], smw[7];
#pragma unroll
                for (int m = 0; m < 7; m++) mx[m] = sm[m] = mxw[m] = smw[m] = 0.f;
                for (int p = lane; p < B.np; p += 32) {
                    float x, y, z, d;
                    if (geo_cached) {
                        const float4 gq = geo[(e - e0) * B.np + p];
                        x = gq.x;
                        y = gq.y;
                        z = gq.z;
                        d = gq.w;
                    } else {
                        const float *pp = P.pts_dd + 6 * (B.pt0 + p);
                        x = (pp[0] + pp[1]) - ax;
                        y = (pp[2] + pp[3]) - ay;
                        z = (pp[4] + pp[5]) - az;
                        d = sqrtf(x * x + y * y + z * z);
                    }
                    const float rad = radial_over_d_f32(R, tab, tstep, d, __frcp_rn(d));
                    if (rad == 0.f) continue;
                    float Q[7];
                    int ci[7];
                    ylm_poly_f32(R.l, x, y, z, Q, ci);
                    const float wvp = wvf[p];
#pragma unroll
                    for (int m = 0; m < 7; m++) {
                        if (m >= nm) break;
                        const float a = fminf(fabsf(rad * kYlmC[ci[m]].x * Q[m]), 1.0e30f);
                        const float aw = fminf(a * wvp, 1.0e30f);
                        mx[m] = fmaxf(mx[m], a);
                        sm[m] += a;
                        mxw[m] = fmaxf(mxw[m], aw);
                        smw[m] += aw;
                    }
                }
#pragma unroll
                for (int m = 0; m < 7; m++) {
                    if (m >= nm) break;
                    unsigned int a = __reduce_max_sync(0xffffffffu, __float_as_uint(mx[m]));
                    unsigned int aw = __reduce_max_sync(0xffffffffu, __float_as_uint(mxw[m]));
                    float s1 = sm[m], s2 = smw[m];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                    }
                    const int fr = f1 + m;
                    if (lane == 0 && fr >= f_lo && fr < f_hi) {
                        const int row = A.fn_loc + fr - r0;
                        rowmax[0][row] = a;
                        rowmax[1][row] = aw;
                        rowsum[0][row] = s1;
                        rowsum[1][row] = s2;
                    }
                }
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < 256; q += blockDim.x) {
            const int which = q >> 7, r = q & 127;
            float sc, un;
            fixed_scale_adaptive(__uint_as_float(rowmax[which][r]), rowsum[which][r], T.nc * 64, sc, un);
            fsc[which][r][0] = sc;
            fsc[which][r][1] = un;
        }
        __syncthreads();
    }
    // the per-point scale of the images: sqrt|w v| (psi) or w v (mixed signs)
    for (int p = threadIdx.x; p < B.np; p += blockDim.x) {
        const double vv = v ? v[B.pt0 + p] : 0.0;
        if (!isfinite(vv)) atomicOr(P.status, kStatusNonFinite);
        const double s = P.pw[B.pt0 + p] * vv;
        df sd = df_from_double(sgn != 0 ? fabs(s) : s);
        if (sgn != 0) sd = df_sqrt(sd);
        wvs[p] = make_float2(sd.hi, sd.lo);
    }
    __syncthreads();
    uint8_t *img1 = sgn == 0 ? a_img : phi_img;
    if (sgn != 0) {
        if (fixed) h_image_lanes<1, 3>(P, B, T, act, sh_tab, I, e0, ne, phi_img, img1, wvs, fsc);
        else h_image_lanes<1, 1>(P, B, T, act, sh_tab, I, e0, ne, phi_img, img1, wvs, fsc);
    } else {
        if (fixed) h_image_lanes<2, 3>(P, B, T, act, sh_tab, I, e0, ne, phi_img, img1, wvs, fsc);
        else h_image_lanes<2, 1>(P, B, T, act, sh_tab, I, e0, ne, phi_img, img1, wvs, fsc);
    }
    // rows past n_b in the last block: zeros (whole 16-byte units)
    const int nlive = rend - r0;
    const int nplanes = fixed ? 3 : 1;
    for (int u = threadIdx.x; u < (128 - nlive) * T.nc * 8; u += blockDim.x) {
        const int r = nlive + u / (T.nc * 8), cg = u % (T.nc * 8);
        const long long off = unit_offset(I, T.nc_alloc, cg >> 3, r, cg & 7);
        for (int pl = 0; pl < nplanes; pl++) {
            *reinterpret_cast<uint4 *>(phi_img + off + pl * T.plane_phi) = make_uint4(0u, 0u, 0u, 0u);
            if (sgn == 0) *reinterpret_cast<uint4 *>(a_img + off + pl * T.plane_phi) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

// CTA per (batch, 64-point chunk c): the phi image for the density.  The
// density contracts over functions, so the fixed-point grid of the leading
// term is per point (column): first the largest |phi_i(p)| over all of the
// batch's functions (FP32), then every 128-row block in double-float.
__global__ void __launch_bounds__(kPhiThreads, 5) k_tc_phi_cols(DevPlan P, const TcBatch *tb, const WorkItem *items,
                                                     uint8_t *ws, int n_split, int bound)
{
    __shared__ unsigned int colmax[64];
    __shared__ float colsum[64];
    __shared__ float csc[2][64];
    __shared__ float ymax[kMaxL + 1];                // max over m of max |Y_lm|, per l
    __shared__ DevShell shs[kMaxShellsSmem];
    const WorkItem it = items[blockIdx.x];
    const DevBatch B = P.batches[it.batch];
    const TcBatch T = tb[it.batch];
    const int c = it.ti;
    const DevAct *act = P.act + B.act0;
    uint8_t *phi_img = ws + T.img_phi;
    const bool fixed = n_split == 3;
    const DevShell *sh_tab = stage_shells(P, shs);
    __syncthreads();
    if (fixed) {
        if (threadIdx.x < 64) {
            colmax[threadIdx.x] = 0u;
            colsum[threadIdx.x] = 0.f;
        }
        if (bound && threadIdx.x <= kMaxL) {
            const int l = threadIdx.x;
            float y = 0.f;
            for (int m = 0; m <= 2 * l; m++) y = fmaxf(y, __ldg(P.rbound + l * l + m));
            ymax[l] = y;
        }
        __syncthreads();
        for (int u = threadIdx.x; u < B.n_act * 64; u += blockDim.x) {
            const int e = u >> 6, k = u & 63, p = c * 64 + k;
            if (p >= B.np) continue;
            const DevAct A = act[e];
            const DevSpecies S = P.species[P.atom_species[A.atom]];
            const float *pp = P.pts_dd + 6 * (B.pt0 + p);
            const float *aa = P.atom_dd + 6 * A.atom;
            const float x = (pp[0] - aa[0]) + (pp[1] - aa[1]);
            const float y = (pp[2] - aa[2]) + (pp[3] - aa[3]);
            const float z = (pp[4] - aa[4]) + (pp[5] - aa[5]);
            const float d = sqrtf(x * x + y * y + z * z);
            if (d > (float)S.rcut * 1.00001f) continue;        // every shell is zero here
            float mx = 0.f, sm = 0.f;
            if (bound) {
                // table bounds: one lookup per shell, the knot index taken
                // from below against FP32 rounding of d
                const float dl = d * 0.999999f;
                for (int sh = 0; sh < S.n_shell; sh++) {
                    const DevShell R = sh_tab[S.shell0 + sh];
                    if (d >= R.rcut_f * 1.00001f) continue;
                    const int ki = min(max((int)(dl * R.inv_h_hi), 0), R.nk - 2);
                    const float tb = __ldg(P.rbound + R.bound_off + ki);
                    mx = fmaxf(mx, fminf(tb * ymax[R.l], 1.0e30f));
                    // sum over m of |Y_lm| <= (2l+1)/sqrt(4 pi): Cauchy-Schwarz with
                    // sum_m Y_lm^2 = (2l+1)/(4 pi) (Unsold's theorem)
                    sm += fminf(tb * (float)(2 * R.l + 1) * (0.28209479f * 1.000001f), 1.0e30f);
                }
                if (!(sm < 1.0e30f)) sm = 1.0e30f;
                atomicMax(&colmax[k], __float_as_uint(mx));
                atomicAdd(&colsum[k], sm);
                continue;
            }
            const float inv_d = __frcp_rn(d);
            for (int sh = 0; sh < S.n_shell; sh++) {
                const DevRadial R = P.radials[P.shell_rad[S.shell0 + sh]];
                int tstep;
                const float4 *tab = spline_tab(P, S, R, sh, tstep);
                const float rad = radial_over_d_f32(R, tab, tstep, d, inv_d);
                float Q[7];
                int ci[7];
                ylm_poly_f32(R.l, x, y, z, Q, ci);
#pragma unroll
                for (int m = 0; m < 7; m++) {
                    if (m >= 2 * R.l + 1) break;
                    const float a = fabsf(rad * kYlmC[ci[m]].x * Q[m]);
                    mx = fmaxf(mx, a);
                    sm += a;
                }
            }
            if (!(mx < 1.0e30f)) mx = 1.0e30f;
            if (!(sm < 1.0e30f)) sm = 1.0e30f;
            atomicMax(&colmax[k], __float_as_uint(mx));
            atomicAdd(&colsum[k], sm);
        }
        __syncthreads();
        if (threadIdx.x < 64) {
            float sc, un;
            fixed_scale_adaptive(__uint_as_float(colmax[threadIdx.x]), colsum[threadIdx.x], T.nkc * 64, sc, un);
            csc[0][threadIdx.x] = sc;
            csc[1][threadIdx.x] = un;
        }
        __syncthreads();
    }
    // warp tasks (active atom, 32-point half of the chunk), lane = point:
    // every function of the atom at the lane's point, split on the point's grid
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int nsplit = fixed ? 3 : 1;
    for (int task = warp; task < B.n_act * 2; task += nwarp) {
        const DevAct A = act[task >> 1];
        const DevSpecies S = P.species[P.atom_species[A.atom]];
        const int k = (task & 1) * 32 + lane, p = c * 64 + k;
        const float *pp = p < B.np ? P.pts_dd + 6 * (B.pt0 + p) : nullptr;
        const float sc = fixed ? csc[0][k] : 0.f, un = fixed ? csc[1][k] : 0.f;
        auto emit = [&](int f, const df *val) {
            const int rg = A.fn_loc + f;
            const int off = elem_offset(rg >> 7, T.nc_alloc, rg & 127, p);
            if (fixed)
                store_value<3>(phi_img + off, T.plane_phi, val[0], sc, un);
            else
                store_value<1>(phi_img + off, T.plane_phi, val[0], sc, un);
        };
        auto emit0 = [&](int f) {
            const int rg = A.fn_loc + f;
            store_zero(phi_img + elem_offset(rg >> 7, T.nc_alloc, rg & 127, p), T.plane_phi, nsplit);
        };
        // the warp's 32 columns of the atom's rows: four 16-byte units per row and plane
        auto zero_all = [&]() {
            const int pc = c * 64 + (task & 1) * 32;
            for (int u = lane; u < S.n_fn * 4; u += 32) {
                const int rg = A.fn_loc + (u >> 2);
                const int off = elem_offset(rg >> 7, T.nc_alloc, rg & 127, pc + (u & 3) * 8);
                for (int pl = 0; pl < nsplit; pl++)
                    *reinterpret_cast<uint4 *>(phi_img + off + pl * T.plane_phi) = make_uint4(0u, 0u, 0u, 0u);
            }
        };
        eval_atom_lane<1, false>(P, S, sh_tab, A.atom, pp, 0, S.n_fn, nullptr, emit, emit0, zero_all);
    }
    // rows [n_b, 64 nkc) of the contraction's last function chunk: zeros
    const int nplanes = fixed ? 3 : 1;
    for (int u = threadIdx.x; u < (T.nkc * 64 - B.nfn) * 8; u += blockDim.x) {
        const int rg = B.nfn + (u >> 3), g = u & 7;
        const long long off = unit_offset(rg >> 7, T.nc_alloc, c, rg & 127, g);
        for (int pl = 0; pl < nplanes; pl++)
            *reinterpret_cast<uint4 *>(phi_img + off + pl * T.plane_phi) = make_uint4(0u, 0u, 0u, 0u);
    }
}

// FP32 value -> signed fixed point with unit 2^-40.  With t = v 2^8,
// h = rint(t) and f = t - h (exact, |f| <= 1/2), the value is
// h 2^32 + trunc(f 2^32): two 32-bit conversions instead of 64-bit shifts.
// The bits below 2^-40 are dropped toward zero (f = +1/2 exactly saturates
// the low word, an error of one unit).  |v| must stay below 2^22; larger or
// non-finite values set *bad.

__device__ __forceinline__ long long f32_to_fix(float v, bool &bad)
{
    const float t = v * 256.f;
    bad |= !(fabsf(t) < 1073741824.f);                 // 2^30; also catches NaN
    const float h = rintf(t);
    const float f = t - h;
    const int hi = __float2int_rz(h);
    const int lo = __float2int_rz(f * 4294967296.f);
    return (long long)hi * 4294967296ll + (long long)lo;
}

// h[k] = (accumulate ? h[k] : 0) + acc[k] 2^-40
__global__ void k_fix_to_h(const long long *acc, double *h, long long n, int accumulate)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double v = (double)acc[k] * 0x1p-40;
        h[k] = accumulate ? h[k] + v : v;
    }
}

// ----------------------------------------------- H contraction on tcgen05 (K2)
// Persistent: one CTA per SM walks the tile list (batch, I, J), I <= J, with
// stride gridDim.x; each tile is 128 x 128 outputs with K = the batch's
// points in chunks of 64, computed transposed (A = phi of block J, B = w v phi
// of block I).  Warp 8 (one lane) streams operand chunks into a two-stage
// shared-memory ring with bulk copies; warp 9 (one lane) issues the MMAs
// into one of two tensor-memory accumulator sets (acc0 + acc1, 256 columns
// each); warps 0-7 drain the other set and scatter the upper triangle into
// the fixed-point H accumulator, so the scatter of one tile overlaps the
// MMAs of the next.  A warp's lanes hold 32 consecutive functions j, so the
// atomics for one column i land on consecutive values of row i.
constexpr int kThreadsTc = 320;                  // warps 0-7 epilogue, 8 producer, 9 MMA
constexpr int kWarpProducer = 8, kWarpMma = 9;
constexpr int kEpiThreads = 256;
constexpr int kStages = 2;
constexpr int kStageBytes = 6 * kChunkBytes;     // A and B operands, 3 planes each
// split products kept in the density: combined order <= 3 except x2*y2 (8 of
// 9), as in H; the order-3 pair x1*y2, x2*y1 is about 2^-27 of the leading
// product, which over ~10^3 functions is no longer far below the 1e-7
// relative bound on n
constexpr int kDensityOrder = 3;

struct ColRef {                                  // column i of an H tile (a row of the stored triangle)
    long long rpl;                               // first stored value of row i minus i's index in its atom
    int atom;                                    // global atom
    int loc;                                     // atom index inside its system
    int slot;                                    // i's atom among the tile's column atoms (0 = first)
    int pad;
};

// Pair offsets of an H tile: for each of the (at most kColAtoms) atoms of
// the tile's columns and each row j, the start of that atom's run in row i
// relative to (rp_i - li), i.e. 0 for j's own atom, pairpos otherwise (-1:
// not stored).  Filled once per tile so that the scatter loop has no
// dependent global loads.
constexpr int kColAtoms = 32;
struct HPairTab {
    int pp[kColAtoms][128];
    int2 atom[2][kColAtoms];                     // (global atom, index in system) per slot
    int nslot[2];
    int pad[2];
};

struct TcRing {
    uint64_t full[kStages], empty[kStages];
    uint64_t tfull[2], tempty[2];
    uint32_t tmem;
    int abort;
    int pad[2];
    ColRef ref[2][128];
};

__device__ __forceinline__ uint8_t *align1024(uint8_t *p)
{
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// named barrier of the eight epilogue warps
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ void ring_init(TcRing *S)
{
    for (int s = 0; s < kStages; s++) {
        mbar_init(&S->full[s], 1);
        mbar_init(&S->empty[s], 1);
    }
    for (int b = 0; b < 2; b++) {
        mbar_init(&S->tfull[b], 1);
        mbar_init(&S->tempty[b], kEpiThreads);
    }
    S->abort = 0;
    fence_mbar_init();
}

// Issue the split products of one 64-deep chunk (4 k-steps of 16): every
// product of combined order <= ORDER except x2*y2; x0*y0 alone in
// accumulator 0.  Fully unrolled with the descriptors of the stage computed
// once: the plane and k-step offsets are added to the descriptors' address
// field (addr >> 4, no carry out of it inside shared memory), so one lane
// issues an MMA every few instructions and keeps the tensor pipe fed.
// first: the chunk opens the item (the first product into each accumulator
// overwrites it).
template <int NSPLIT, int ORDER, bool B_MN>
__device__ __forceinline__ void mma_chunk(uint32_t acc_base, const uint8_t *a_sm, const uint8_t *b_sm, uint32_t idesc,
                                          bool first)
{
    const uint64_t ad0 = desc_sw128(smem_u32(a_sm), 16, 1024);
    const uint64_t bd0 = B_MN ? desc_sw128(smem_u32(b_sm), 8192, 1024) : desc_sw128(smem_u32(b_sm), 16, 1024);
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
#pragma unroll
        for (int pa = 0; pa < NSPLIT; pa++) {
#pragma unroll
            for (int pb = 0; pb < NSPLIT; pb++) {
                if (pa + pb > ORDER || (pa == 2 && pb == 2)) continue;
                const int acc = (pa + pb == 0) ? 0 : 1;
                const uint64_t ad = ad0 + (uint64_t)((pa * kChunkBytes + ks * 32) >> 4);
                const uint64_t bd = bd0 + (uint64_t)((pb * kChunkBytes + ks * (B_MN ? 2048 : 32)) >> 4);
                const bool opens = ks == 0 && (acc == 0 || (pa == 0 && pb == 1));
                tc_mma(acc_base + acc * 128, ad, bd, idesc, (first && opens) ? 0u : 1u);
            }
        }
    }
}

__global__ void __launch_bounds__(kThreadsTc, 1) k_tc_h(DevPlan P, const TcBatch *tb, const WorkItem *items,
                                                        int n_items, const uint8_t *ws, unsigned long long *hfix,
                                                        int n_split, const int *bsign)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1024(smem_raw);
    TcRing *S = reinterpret_cast<TcRing *>(sm + kStages * kStageBytes);
    HPairTab *PT = reinterpret_cast<HPairTab *>(
        (reinterpret_cast<uintptr_t>(S + 1) + 15) & ~(uintptr_t)15);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) ring_init(S);
    if (warp == kWarpMma) {
        tmem_alloc(&S->tmem, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S->tmem;
    const uint32_t chunk = (uint32_t)n_split * kChunkBytes;

    if (warp == kWarpProducer) {
        if (lane == 0) {
            long long n = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_items && ok; t += gridDim.x) {
                const WorkItem it = items[t];
                const TcBatch T = tb[it.batch];
                // A = phi rows of block J (TMEM lanes), B = w v phi rows of block I
                // (TMEM columns): the transposed tile, so that the scatter of one
                // column i by the 32 lanes of a warp hits consecutive values of row i.
                // Batches where w v has one sign hold psi = phi sqrt|w v| in the
                // phi image, which then serves as both operands.
                const uint8_t *a_img = ws + T.img_phi;
                const uint8_t *b_img = ws + (bsign[it.batch] != 0 ? T.img_phi : T.img_aux);
                for (int c = 0; c < T.nc; c++, n++) {
                    const int st = (int)(n % kStages);
                    const long long use = n / kStages;
                    if (use > 0 && !mbar_wait_a(&S->empty[st], (uint32_t)((use - 1) & 1), P.status, &S->abort)) {
                        ok = false;
                        break;
                    }
                    uint8_t *a_sm = sm + st * kStageBytes, *b_sm = a_sm + 3 * kChunkBytes;
                    mbar_expect_tx(&S->full[st], 2 * chunk);
                    for (int s = 0; s < n_split; s++) {
                        bulk_g2s(a_sm + s * kChunkBytes,
                                 a_img + s * T.plane_phi + (long long)(it.tj * T.nc_alloc + c) * kChunkBytes,
                                 kChunkBytes, &S->full[st]);
                        bulk_g2s(b_sm + s * kChunkBytes,
                                 b_img + s * T.plane_phi + (long long)(it.ti * T.nc_alloc + c) * kChunkBytes,
                                 kChunkBytes, &S->full[st]);
                    }
                }
            }
            // do not leave while a copy may still be landing
            for (long long q = (n > kStages ? n - kStages : 0); q < n; q++)
                mbar_wait_a(&S->empty[q % kStages], (uint32_t)((q / kStages) & 1), P.status, &S->abort);
        }
        __syncwarp();
    } else if (warp == kWarpMma) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(128, 128, false, false);
            long long n = 0;
            int lt = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_items && ok; t += gridDim.x, lt++) {
                const TcBatch T = tb[items[t].batch];
                const int buf = lt & 1, use = lt >> 1;
                if (use > 0 && !mbar_wait_a(&S->tempty[buf], (uint32_t)((use - 1) & 1), P.status, &S->abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int c = 0; c < T.nc; c++, n++) {
                    const int st = (int)(n % kStages);
                    if (!mbar_wait_a(&S->full[st], (uint32_t)((n / kStages) & 1), P.status, &S->abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint8_t *a_sm = sm + st * kStageBytes;
                    if (n_split == 3)
                        mma_chunk<3, 3, false>(tmem + buf * 256, a_sm, a_sm + 3 * kChunkBytes, idesc, c == 0);
                    else
                        mma_chunk<1, 0, false>(tmem + buf * 256, a_sm, a_sm + 3 * kChunkBytes, idesc, c == 0);
                    tc_commit(&S->empty[st]);
                }
                tc_commit(&S->tfull[buf]);
            }
        }
        __syncwarp();
    } else {
        // epilogue warp w: TMEM lanes 32 (w % 4) .. + 31 (functions j of block J),
        // columns 64 (w / 4) .. + 63 (functions i of block I)
        int lt = 0;
        bool bad = false;
        const int quad = warp & 3, half = warp >> 2;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        for (int t = blockIdx.x; t < n_items; t += gridDim.x, lt++) {
            const WorkItem it = items[t];
            const DevBatch B = P.batches[it.batch];
            const DevAct *act = P.act + B.act0;
            const int buf = lt & 1, use = lt >> 1;
            const int i0 = it.ti * 128, j0 = it.tj * 128;
            const int *pp_sys = P.pairpos + P.sys_pair_off[B.sys];
            const int nat = P.sys_nat[B.sys];
            if (threadIdx.x < 128) {
                const int i = i0 + threadIdx.x;
                const int ilast = min(i0 + 127, B.nfn - 1);
                if (i <= ilast) {
                    const int e_first = find_act(act, B.n_act, i0);
                    const int e = find_act(act, B.n_act, i);
                    const FnRef c = fn_ref(P, act, e, i);
                    const int slot = e - e_first;
                    S->ref[buf][threadIdx.x] = ColRef{c.rp - c.li, c.atom, c.loc, slot, 0};
                    if (slot < kColAtoms && (i == i0 || act[e].fn_loc == i))
                        PT->atom[buf][slot] = make_int2(c.atom, c.loc);
                    if (i == ilast) PT->nslot[buf] = slot + 1;
                } else {
                    S->ref[buf][threadIdx.x] = ColRef{0, -1, 0, 0, 0};   // past the batch: a valid slot, never stored
                }
            }
            const int r = quad * 32 + lane;
            const int j = j0 + r;                  // this lane's function (block J)
            FnRef jref{};
            if (j < B.nfn) jref = fn_ref(P, act, find_act(act, B.n_act, j), j);
            const bool negate = bsign[it.batch] < 0;            // H = -psi^T psi
            epi_sync();
            // pair offsets of this tile (the previous tile's scatter is over)
            const int nslot = PT->nslot[buf];
            const bool tab = nslot <= kColAtoms;
            if (tab && j < B.nfn) {
                for (int sl = half; sl < nslot; sl += 2) {
                    const int2 a = PT->atom[buf][sl];
                    PT->pp[sl][r] = a.x == jref.atom ? 0 : __ldg(pp_sys + (long long)a.y * nat + jref.loc);
                }
            }
            epi_sync();
            const bool ok = mbar_wait_a(&S->tfull[buf], (uint32_t)(use & 1), P.status, &S->abort);
            tc_fence_after();
            const uint32_t acc_base = tmem + buf * 256 + lane_base;
            for (int cq = 0; cq < 2; cq++) {
                const int cc = 2 * half + cq;
                if (i0 + cc * 32 >= B.nfn) break;
                float a0[32], a1[32];
                tmem_ld32(acc_base + cc * 32, a0);
                if (n_split > 1) tmem_ld32(acc_base + 128 + cc * 32, a1);
                tmem_wait_ld();
                if (!ok || j >= B.nfn) continue;
                // stored value of (i, j), i <= j: row i, (rp_i - li) + [pair offset of
                // atom(j) in row i, 0 for the same atom] + lj
                unsigned long long *hj = hfix + jref.li;
                if (tab) {
                    // branch-free per column (predicated atomics), so the conversions
                    // of neighbouring columns overlap
#pragma unroll
                    for (int q = 0; q < 32; q++) {
                        const int il = cc * 32 + q;
                        const int i = i0 + il;
                        const long long rpl = S->ref[buf][il].rpl;
                        const int ppv = PT->pp[S->ref[buf][il].slot][r];
                        long long fx = f32_to_fix(a0[q], bad);
                        if (n_split > 1) fx += f32_to_fix(a1[q], bad);
                        if (negate) fx = -fx;
                        if (i < B.nfn && i <= j && ppv >= 0 && fx != 0)
                            atomicAdd(hj + rpl + ppv, (unsigned long long)fx);
                    }
                    continue;
                }
                int cur_atom = -1;                 // more column atoms than table slots
                int ppv = 0;
                bool stored = false;
#pragma unroll
                for (int q = 0; q < 32; q++) {
                    const int il = cc * 32 + q;
                    const int i = i0 + il;
                    if (i >= B.nfn || i > j) continue;
                    const ColRef ci = S->ref[buf][il];
                    if (ci.atom != cur_atom) {
                        cur_atom = ci.atom;
                        if (ci.atom == jref.atom) {
                            ppv = 0;
                            stored = true;
                        } else {
                            ppv = __ldg(pp_sys + (long long)ci.loc * nat + jref.loc);
                            stored = ppv >= 0;
                        }
                    }
                    if (!stored) continue;
                    long long fx = f32_to_fix(a0[q], bad);
                    if (n_split > 1) fx += f32_to_fix(a1[q], bad);
                    if (negate) fx = -fx;
                    if (fx != 0) atomicAdd(hj + ci.rpl + ppv, (unsigned long long)fx);
                }
            }
            tc_fence_before();
            mbar_arrive(&S->tempty[buf]);
        }
        if (bad) atomicOr(P.status, kStatusNonFinite);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kWarpMma) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------- D_b gather (K3a)
// CTA per (batch, 128-row block J): D(j, i) for local functions j (rows) and
// i (columns) from the stored upper triangle, split into BF16 planes as a
// K-major swizzled image.  In the split mode the leading term is fixed-point
// on a per-row grid (the density contracts over i), found by a first pass
// over the row block.
// D values as double-floats (once per density call; nnz elements), and for
// every function g the largest |D_gi| and the sum of |D_gi| over its full
// symmetric row: bounds (valid for every batch) for the fixed-point grid of
// the gathered rows.  One warp per row of the stored upper triangle.
__global__ void k_to_df(const double *x, float2 *out, const long long *rowptr, const int *fn_sys,
                        const long long *sys_val0, const long long *sys_nnz, long long n_fn, unsigned int *gmax,
                        float *gsum)
{
    const int lane = threadIdx.x & 31;
    const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g = warp0; g < n_fn; g += nwarps) {
        const int s = fn_sys[g];
        const long long k0 = rowptr[g];
        const long long k1 = (g + 1 < n_fn && fn_sys[g + 1] == s) ? rowptr[g + 1] : sys_val0[s] + sys_nnz[s];
        float mx = 0.f, sm = 0.f;
        for (long long k = k0 + lane; k < k1; k += 32) {
            const df v = df_from_double(x[k]);
            out[k] = make_float2(v.hi, v.lo);
            float a = fabsf(v.hi);
            if (!(a < 1.0e30f)) a = 1.0e30f;
            mx = fmaxf(mx, a);
            sm += a;
        }
        mx = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
        if (lane == 0) {
            atomicMax(gmax + g, __float_as_uint(mx));
            atomicAdd(gsum + g, sm);
        }
    }
}

constexpr int kGatherActSmem = 512;     // active atoms of a batch the gather stages in shared memory

// the column side of the symmetric rows: value (g, j), j > g, bounds row j
__global__ void k_d_colbounds(const float2 *v, const int *col_of, long long nnz, unsigned int *gmax, float *gsum)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x) {
        const int j = col_of[k];
        if (j < 0) continue;                       // diagonal entries are counted once
        float a = fabsf(v[k].x);
        if (!(a < 1.0e30f)) a = 1.0e30f;
        atomicMax(gmax + j, __float_as_uint(a));
        atomicAdd(gsum + j, a);
    }
}

__global__ void __launch_bounds__(256) k_tc_gather_d(DevPlan P, const TcBatch *tb, const WorkItem *items,
                                                     uint8_t *ws, const float2 *ddv, const unsigned int *gmax,
                                                     const float *gsum, float offdiag_scale, int n_split, int full)
{
    const WorkItem it = items[blockIdx.x];
    const DevBatch B = P.batches[it.batch];
    const TcBatch T = tb[it.batch];
    const int J = it.ti;
    __shared__ FnRef rref[128], cref[64];
    __shared__ float rsc[2][128];
    __shared__ int4 sact[kGatherActSmem];            // per active atom: fn_loc, atom, loc, first global fn
    const DevAct *act = P.act + B.act0;
    const bool fixed = n_split == 3;
    const int *pp_sys = P.pairpos + P.sys_pair_off[B.sys];
    const int nat = P.sys_nat[B.sys];
    // the batch's active atoms in shared memory, so that each column's
    // reference costs one search there and one global load (its row start)
    const bool staged = B.n_act <= kGatherActSmem;
    if (staged) {
        for (int e = threadIdx.x; e < B.n_act; e += blockDim.x) {
            const DevAct A = act[e];
            sact[e] = make_int4(A.fn_loc, A.atom, P.atom_loc[A.atom], (int)P.atom_fn0[A.atom]);
        }
    }
    __syncthreads();
    auto ref_of = [&](int l) -> FnRef {
        if (!staged) return fn_ref(P, act, find_act(act, B.n_act, l), l);
        int lo = 0, hi = B.n_act - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sact[mid].x <= l) lo = mid; else hi = mid - 1;
        }
        const int4 a = sact[lo];
        FnRef r;
        r.atom = a.y;
        r.li = l - a.x;
        r.gi = (long long)a.w + r.li;
        r.rp = __ldg(P.rowptr + r.gi);
        r.loc = a.z;
        r.pad = 0;
        return r;
    };
    if (threadIdx.x < 128) {
        const int j = J * 128 + threadIdx.x;
        float sc = 0.f, un = 0.f;
        if (j < B.nfn) {
            const FnRef rj = ref_of(j);
            rref[threadIdx.x] = rj;
            if (fixed) fixed_scale_adaptive(__uint_as_float(gmax[rj.gi]), gsum[rj.gi], T.nkc * 64, sc, un);
        }
        rsc[0][threadIdx.x] = sc;
        rsc[1][threadIdx.x] = un;
    }
    uint8_t *img = ws + T.img_aux;
    // D is symmetric: block row J holds only the chunks i >= 128 J, the
    // diagonal block halved (n = 2 sum_J phi_J . E_J, exact in binary); in
    // full (the adjoint's G Phi) every chunk, nothing halved
    for (int kc = full ? 0 : 2 * J; kc < T.nkc; kc++) {
        const float blk = (!full && kc < 2 * J + 2) ? 0.5f : 1.f;
        __syncthreads();
        if (threadIdx.x < 64) {
            const int i = kc * 64 + threadIdx.x;
            if (i < B.nfn) cref[threadIdx.x] = ref_of(i);
        }
        __syncthreads();
        for (int u = threadIdx.x; u < 1024; u += blockDim.x) {
            const int r = u >> 3, g = u & 7;
            const int j = J * 128 + r;
            const FnRef rj = rref[r];
            // stored value of (j, i): for i >= j, base + gi (row j's run of atom(i));
            // for i < j, rp_i - li + off (row i's run of atom(j)); cached per column atom
            int cur_atom = -1;
            long long off = 0;
            bool stored = false;
            df x[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int il = g * 8 + q;
                const int i = kc * 64 + il;
                x[q] = df{0.f, 0.f};
                if (j >= B.nfn || i >= B.nfn) continue;
                const FnRef &ci = cref[il];
                if (ci.atom != cur_atom) {
                    cur_atom = ci.atom;
                    if (ci.atom == rj.atom) {
                        stored = true;
                        off = 0;
                    } else if (ci.atom > rj.atom) {
                        const int pp = __ldg(pp_sys + (long long)rj.loc * nat + ci.loc);
                        stored = pp >= 0;
                        off = rj.rp + pp - rj.li - (ci.gi - ci.li);       // + gi
                    } else {
                        const int pp = __ldg(pp_sys + (long long)ci.loc * nat + rj.loc);
                        stored = pp >= 0;
                        off = pp + rj.li;                                   // + rp_i - li
                    }
                }
                if (!stored) continue;
                long long k;
                if (ci.atom == rj.atom)
                    k = i >= j ? rj.rp + (ci.gi - rj.gi) : ci.rp + (rj.gi - ci.gi);
                else
                    k = ci.atom > rj.atom ? off + ci.gi : ci.rp - ci.li + off;
                const float2 v = __ldg(ddv + k);
                const float sc = (i == j ? 1.f : offdiag_scale) * blk;
                x[q] = df{v.x * sc, v.y * sc};
            }
            uint8_t *dst = img + unit_offset(J, T.nkc, kc, r, g);
            if (fixed)
                store_fixed8(dst, T.plane_d, x, rsc[0][r], rsc[1][r]);
            else
                store_split8_df(dst, T.plane_d, x, n_split);
        }
    }
}

// ------------------------------------------------- density on tcgen05 (K3b)
// Persistent: one CTA per SM walks the items (batch, 128-point tile m,
// 128-function block J), J ascending so the longest contractions come first:
// E^T[j][p] = sum_{i >= 128 J} D'[j][i] phi_i(p) over the upper block
// triangle of the symmetric D (D' = D with its diagonal block halved;
// A = D image, K-major; B = phi image read as MN-major) accumulates in one of
// two tensor-memory sets while warps 0-7 finish the previous item: the
// partial density sum_{j in J} E^T[j][p] phi_j(p) in double-float (lane j
// multiplies by its own phi row, the warp reduces over j), one row of 128
// doubles per item.  Many items per batch keep the CTAs on few batches at a
// time, so the D and phi images are read from L2.  k_density_sum then forms
// n_p = 2 sum_J partial_J(p).
//
// ADJ (the adjoint's E = G Phi): every function chunk of the full G image,
// and each lane also stores its row of E (acc0 + acc1 in FP32) for the
// position gradient.
template <bool ADJ>
__global__ void __launch_bounds__(kThreadsTc, 1) k_tc_density(DevPlan P, const TcBatch *tb, const WorkItem *items,
                                                              int n_items, const uint8_t *ws, double *part,
                                                              int n_split, uint8_t *ws_e)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1024(smem_raw);
    TcRing *S = reinterpret_cast<TcRing *>(sm + kStages * kStageBytes);
    __shared__ double red[4][128];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) ring_init(S);
    if (warp == kWarpMma) {
        tmem_alloc(&S->tmem, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S->tmem;
    const uint32_t chunk = (uint32_t)n_split * kChunkBytes;

    if (warp == kWarpProducer) {
        if (lane == 0) {
            long long n = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_items && ok; t += gridDim.x) {
                const WorkItem it = items[t];
                const TcBatch T = tb[it.batch];
                const int m = it.ti, J = it.tj;
                const uint8_t *d_img = ws + T.img_aux, *phi_img = ws + T.img_phi;
                for (int kc = ADJ ? 0 : 2 * J; kc < T.nkc; kc++, n++) {
                    const int st = (int)(n % kStages);
                    const long long use = n / kStages;
                    if (use > 0 && !mbar_wait_a(&S->empty[st], (uint32_t)((use - 1) & 1), P.status, &S->abort)) {
                        ok = false;
                        break;
                    }
                    uint8_t *a_sm = sm + st * kStageBytes, *b_sm = a_sm + 3 * kChunkBytes;
                    mbar_expect_tx(&S->full[st], 2 * chunk);
                    const int I = kc >> 1, half = kc & 1;
                    for (int s = 0; s < n_split; s++) {
                        bulk_g2s(a_sm + s * kChunkBytes,
                                 d_img + s * T.plane_d + (long long)(J * T.nkc + kc) * kChunkBytes, kChunkBytes,
                                 &S->full[st]);
                        for (int c2 = 0; c2 < 2; c2++)
                            bulk_g2s(b_sm + s * kChunkBytes + c2 * 8192,
                                     phi_img + s * T.plane_phi +
                                         ((long long)(I * T.nc_alloc + 2 * m + c2) * 16 + 8 * half) * 1024,
                                     8192, &S->full[st]);
                    }
                }
            }
            for (long long q = (n > kStages ? n - kStages : 0); q < n; q++)
                mbar_wait_a(&S->empty[q % kStages], (uint32_t)((q / kStages) & 1), P.status, &S->abort);
        }
        __syncwarp();
    } else if (warp == kWarpMma) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(128, 128, false, true);
            long long n = 0;
            int u = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_items && ok; t += gridDim.x, u++) {
                const WorkItem it = items[t];
                const TcBatch T = tb[it.batch];
                const int J = it.tj;
                const int buf = u & 1, use = u >> 1;
                if (use > 0 && !mbar_wait_a(&S->tempty[buf], (uint32_t)((use - 1) & 1), P.status, &S->abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int kc0 = ADJ ? 0 : 2 * J;
                for (int kc = kc0; kc < T.nkc; kc++, n++) {
                    const int st = (int)(n % kStages);
                    if (!mbar_wait_a(&S->full[st], (uint32_t)((n / kStages) & 1), P.status, &S->abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint8_t *a_sm = sm + st * kStageBytes;
                    if (n_split == 3)
                        mma_chunk<3, kDensityOrder, true>(tmem + buf * 256, a_sm, a_sm + 3 * kChunkBytes, idesc,
                                                          kc == kc0);
                    else
                        mma_chunk<1, 0, true>(tmem + buf * 256, a_sm, a_sm + 3 * kChunkBytes, idesc, kc == kc0);
                    tc_commit(&S->empty[st]);
                }
                tc_commit(&S->tfull[buf]);
            }
        }
        __syncwarp();
    } else {
        // epilogue warp w: TMEM lanes 32 (w % 4) .. + 31 (functions j of the
        // block), point columns 64 (w / 4) .. + 63
        const int quad = warp & 3, half = warp >> 2;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        int u = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < n_items; t += gridDim.x, u++) {
            const WorkItem it = items[t];
            const DevBatch B = P.batches[it.batch];
            const TcBatch T = tb[it.batch];
            const int m = it.ti, J = it.tj;
            const uint8_t *phi_img = ws + T.img_phi;
            const int buf = u & 1, use = u >> 1;
            const int r = quad * 32 + lane;
            const int j = J * 128 + r;
            // this warp's phi rows for the first of its two column chunks: issued
            // before the wait so the loads overlap the MMAs
            uint4 pre[3][4];
            {
                const int cc = 2 * half, c = 2 * m + (cc >> 1);
#pragma unroll
                for (int gg = 0; gg < 4; gg++) {
                    const long long off = unit_offset(J, T.nc_alloc, c, r, (cc & 1) * 4 + gg);
#pragma unroll
                    for (int sp = 0; sp < 3; sp++)
                        pre[sp][gg] = sp < n_split ? *reinterpret_cast<const uint4 *>(phi_img + off + sp * T.plane_phi)
                                                   : make_uint4(0u, 0u, 0u, 0u);
                }
            }
            ok = mbar_wait_a(&S->tfull[buf], (uint32_t)(use & 1), P.status, &S->abort);
            tc_fence_after();
            const uint32_t acc_base = tmem + buf * 256 + lane_base;
            for (int cq = 0; cq < 2; cq++) {
                const int cc = 2 * half + cq;
                float a0[32], a1[32];
                tmem_ld32(acc_base + cc * 32, a0);
                if (n_split > 1)
                    tmem_ld32(acc_base + 128 + cc * 32, a1);
                else
#pragma unroll
                    for (int q = 0; q < 32; q++) a1[q] = 0.f;
                tmem_wait_ld();
                if (cq == 1) {
                    tc_fence_before();
                    mbar_arrive(&S->tempty[buf]);     // accumulator set may be reused
                }
                // E^T[j][p] phi_j(p) for the 32 points of this column chunk in
                // double-float (FP32 pipe): e = acc0 + acc1, phi = sum of its planes
                const int c = 2 * m + (cc >> 1);
                const bool live = ok && j < B.nfn;
                if (ADJ && live) {
                    // this lane's row of E at the chunk's 32 points, for the gradient
                    float4 *dst = reinterpret_cast<float4 *>(ws_e + T.img_e) +
                                  ((long long)j * T.nc_alloc * 64 + m * 128 + cc * 32) / 4;
#pragma unroll
                    for (int q4 = 0; q4 < 8; q4++)
                        dst[q4] = make_float4(a0[4 * q4] + a1[4 * q4], a0[4 * q4 + 1] + a1[4 * q4 + 1],
                                              a0[4 * q4 + 2] + a1[4 * q4 + 2], a0[4 * q4 + 3] + a1[4 * q4 + 3]);
                }
#pragma unroll
                for (int gg = 0; gg < 4; gg++) {
                    const int g = (cc & 1) * 4 + gg;
                    const long long off = unit_offset(J, T.nc_alloc, c, r, g);
                    uint32_t w[3][4] = {};
#pragma unroll
                    for (int sp = 0; sp < 3; sp++) {
                        uint4 uu;
                        if (cq == 0)
                            uu = pre[sp][gg];
                        else
                            uu = sp < n_split ? *reinterpret_cast<const uint4 *>(phi_img + off + sp * T.plane_phi)
                                              : make_uint4(0u, 0u, 0u, 0u);
                        w[sp][0] = uu.x; w[sp][1] = uu.y; w[sp][2] = uu.z; w[sp][3] = uu.w;
                    }
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int col = gg * 8 + q;
                        const float f0 = __uint_as_float((q & 1) ? (w[0][q >> 1] & 0xFFFF0000u) : (w[0][q >> 1] << 16));
                        const float f1 = __uint_as_float((q & 1) ? (w[1][q >> 1] & 0xFFFF0000u) : (w[1][q >> 1] << 16));
                        const float f2 = __uint_as_float((q & 1) ? (w[2][q >> 1] & 0xFFFF0000u) : (w[2][q >> 1] << 16));
                        df ph = df_two_sum(f0, f1);
                        ph = df_fast_two_sum(ph.hi, ph.lo + f2);
                        const df e = df_two_sum(a0[col], n_split > 1 ? a1[col] : 0.f);
                        const df pr = df_mul(e, ph);
                        a0[col] = live ? pr.hi : 0.f;
                        a1[col] = live ? pr.lo : 0.f;
                    }
                }
                // reduce over the 32 lanes (rows j): lane q ends with column q
#pragma unroll
                for (int wd = 16; wd >= 1; wd >>= 1) {
                    const bool upper = (lane & wd) != 0;
#pragma unroll
                    for (int q = 0; q < wd; q++) {
                        const float sh = upper ? a0[q] : a0[q + wd], sl = upper ? a1[q] : a1[q + wd];
                        const float kh = upper ? a0[q + wd] : a0[q], kl = upper ? a1[q + wd] : a1[q];
                        const df rcv{__shfl_xor_sync(0xffffffffu, sh, wd), __shfl_xor_sync(0xffffffffu, sl, wd)};
                        const df sum = df_add(df{kh, kl}, rcv);
                        a0[q] = sum.hi;
                        a1[q] = sum.lo;
                    }
                }
                red[quad][cc * 32 + lane] = (double)a0[0] + (double)a1[0];
            }
            // item complete: this block's partial density at the tile's 128 points
            epi_sync();
            if (threadIdx.x < 128) {
                const long long row = T.part0 + (long long)J * (T.nc_alloc / 2) + m;
                part[row * 128 + threadIdx.x] =
                    ok ? (red[0][threadIdx.x] + red[1][threadIdx.x]) + (red[2][threadIdx.x] + red[3][threadIdx.x])
                       : 0.0;
            }
            epi_sync();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kWarpMma) tmem_dealloc(tmem, 512);
}

// n_p = 2 sum_J part[J][p] over the batch's function blocks, in J order
// (deterministic); one CTA of 128 threads per (batch, point tile).
__global__ void __launch_bounds__(128) k_density_sum(DevPlan P, const TcBatch *tb, const WorkItem *items,
                                                    const double *part, double *n_out, double factor)
{
    const WorkItem it = items[blockIdx.x];
    const DevBatch B = P.batches[it.batch];
    const TcBatch T = tb[it.batch];
    const int p = it.ti * 128 + threadIdx.x;
    if (p >= B.np) return;
    const long long nt = T.nc_alloc / 2;
    double s = 0.0;
    for (int J = 0; J < T.nrb; J++) s += part[(T.part0 + J * nt + it.ti) * 128 + threadIdx.x];
    n_out[B.pt0 + p] = factor * s;
}

// sum over the shell's 2l+1 functions of E_i grad phi_i (FP32), unrolled per l
template <int L>
__device__ __forceinline__ void adj_shell(float g, float gp, float x, float y, float z, float nx, float ny, float nz,
                                          const float *Erow, long long Pa, float &gx, float &gy, float &gz)
{
    float Y[2 * L + 1], G[2 * L + 1][3];
    ylm_unit<float>(L, x, y, z, Y);                      // P(r) = r^l Y_lm
    ylm_poly_grad<float>(L, x, y, z, G);
#pragma unroll
    for (int m = 0; m < 2 * L + 1; m++) {
        const float e = __ldg(Erow + m * Pa);
        const float a = gp * Y[m];
        gx = fmaf(e, fmaf(a, nx, g * G[m][0]), gx);
        gy = fmaf(e, fmaf(a, ny, g * G[m][1]), gy);
        gz = fmaf(e, fmaf(a, nz, g * G[m][2]), gz);
    }
}

// Position gradient of the adjoint on CUDA cores (FP32): CTA per (batch,
// 64-point chunk); warp tasks (active atom, 32-point half), lane = point.
// The lane forms sum_{i on the atom} grad phi_i(p) . E_i(p) from the E rows
// the contraction stored, times -2 w_p v_p; the warp sums its 32 points and
// adds the atom's three components to dR (FP64 atomics).
//   grad phi = g'(d) (r/d) P(r) + g(d) grad P(r),  g = u/d^(l+1),
//   g' = u'/d^(l+1) - (l+1) u/d^(l+2),  P = r^l Y_lm (a polynomial in x, y, z)
__global__ void __launch_bounds__(256) k_tc_adj_grad(DevPlan P, const TcBatch *tb, const WorkItem *items,
                                                     const uint8_t *ws, const double *v, double *dR)
{
    const WorkItem it = items[blockIdx.x];
    const DevBatch B = P.batches[it.batch];
    const TcBatch T = tb[it.batch];
    const int c = it.ti;
    const DevAct *act = P.act + B.act0;
    const float *E = reinterpret_cast<const float *>(ws + T.img_e);
    const long long Pa = (long long)T.nc_alloc * 64;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int task = warp; task < B.n_act * 2; task += nwarp) {
        const DevAct A = act[task >> 1];
        const int p = c * 64 + (task & 1) * 32 + lane;
        float gx = 0.f, gy = 0.f, gz = 0.f;
        if (p < B.np) {
            const DevSpecies S = P.species[P.atom_species[A.atom]];
            const float *pp = P.pts_dd + 6 * (B.pt0 + p);
            const float *aa = P.atom_dd + 6 * A.atom;
            const float x = (pp[0] - aa[0]) + (pp[1] - aa[1]);
            const float y = (pp[2] - aa[2]) + (pp[3] - aa[3]);
            const float z = (pp[4] - aa[4]) + (pp[5] - aa[5]);
            const float d = sqrtf(x * x + y * y + z * z);
            if (d > 1e-12f && d < (float)S.rcut * 1.00001f) {
                const float inv = 1.f / d;
                const float nx = x * inv, ny = y * inv, nz = z * inv;
                int f = 0;
                for (int sh = 0; sh < S.n_shell; sh++) {
                    const DevRadial R = P.radials[P.shell_rad[S.shell0 + sh]];
                    const int nm = 2 * R.l + 1;
                    if (d >= R.rcut_f) {
                        f += nm;
                        continue;
                    }
                    const float s = d * R.inv_h_hi;
                    const int k = min((int)s, R.nk - 2);
                    const float t = s - (float)k;
                    const float4 ch = __ldg(P.coef_dd + 2 * (R.coef_off + k));
                    const float u = ch.x + t * (ch.y + t * (ch.z + t * ch.w));
                    const float du = (ch.y + t * (2.f * ch.z + 3.f * t * ch.w)) * R.inv_h_hi;
                    float ipl = inv;
                    for (int q = 0; q < R.l; q++) ipl *= inv;          // 1/d^(l+1)
                    const float g = u * ipl;
                    const float gp = (du - (float)(R.l + 1) * u * inv) * ipl;
                    const float *Erow = E + (long long)(A.fn_loc + f) * Pa + p;
                    switch (R.l) {
                    case 0: adj_shell<0>(g, gp, x, y, z, nx, ny, nz, Erow, Pa, gx, gy, gz); break;
                    case 1: adj_shell<1>(g, gp, x, y, z, nx, ny, nz, Erow, Pa, gx, gy, gz); break;
                    case 2: adj_shell<2>(g, gp, x, y, z, nx, ny, nz, Erow, Pa, gx, gy, gz); break;
                    default: adj_shell<3>(g, gp, x, y, z, nx, ny, nz, Erow, Pa, gx, gy, gz); break;
                    }
                    f += nm;
                }
                const float pref = (float)(-2.0 * P.pw[B.pt0 + p] * v[B.pt0 + p]);
                gx *= pref;
                gy *= pref;
                gz *= pref;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
            gz += __shfl_xor_sync(0xffffffffu, gz, o);
        }
        if (lane == 0 && (gx != 0.f || gy != 0.f || gz != 0.f)) {
            atomicAdd(dR + 3 * A.atom + 0, (double)gx);
            atomicAdd(dR + 3 * A.atom + 1, (double)gy);
            atomicAdd(dR + 3 * A.atom + 2, (double)gz);
        }
    }
}

// Dynamic shared memory of the tcgen05 kernels: the two-stage ring (about
// 200 KB) keeps one CTA per SM, which holds all 512 tensor-memory columns.
size_t smem_tc(int n_split)
{
    (void)n_split;
    return 1024 + (size_t)kStages * kStageBytes + sizeof(TcRing);
}

size_t smem_phi() { return 128 * kPhiValStride * sizeof(float2); }

size_t smem_tc_h() { return smem_tc(3) + sizeof(HPairTab) + 16; }

bool attrs_set = false;

cudaError_t set_attrs()
{
    if (attrs_set) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_tc_h, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_tc_h());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_density<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_tc(3));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_density<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_tc(3));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_phi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_phi());
    if (e != cudaSuccess) return e;
    attrs_set = true;
    return cudaSuccess;
}

}  // namespace

// ==================================================================== host
// Super-batches: runs of consecutive batches of one system (the batcher
// emits spatial neighbours consecutively), merged while the points stay
// within sb_points and the union of active atoms carries at most
// sb_growth times the functions of the largest member.  Every sum of the
// method is over points, so any grouping of points gives the same H and n;
// merging cuts the per-batch scatter, D gather and tile overheads.
static void build_super_batches(TcPlan &t, const TcPlanInput &in, int sb_points, double sb_growth)
{
    t.sb.clear();
    t.sact.clear();
    t.sb_first.clear();
    std::vector<int> uni, tmp;
    int b = 0;
    while (b < in.n_batch) {
        t.sb_first.push_back(b);
        const DevBatch &B0 = in.batches[b];
        uni.clear();
        for (int e = 0; e < B0.n_act; e++) uni.push_back(in.act[B0.act0 + e].atom);
        int np = B0.np, maxfn = B0.nfn, b2 = b + 1;
        while (sb_points > 0 && b2 < in.n_batch && in.batches[b2].sys == B0.sys &&
               np + in.batches[b2].np <= sb_points) {
            const DevBatch &Bn = in.batches[b2];
            tmp.clear();
            size_t i = 0;
            int e = 0;
            while (i < uni.size() || e < Bn.n_act) {
                const int a = e < Bn.n_act ? in.act[Bn.act0 + e].atom : 1 << 30;
                const int u = i < uni.size() ? uni[i] : 1 << 30;
                if (u == a) { tmp.push_back(u); i++; e++; }
                else if (u < a) { tmp.push_back(u); i++; }
                else { tmp.push_back(a); e++; }
            }
            long long nfn = 0;
            for (int a : tmp) nfn += in.atom_nfn[a];
            const int mx = std::max(maxfn, Bn.nfn);
            if (nfn > sb_growth * mx || nfn > kMaxBatchFns) break;
            uni.swap(tmp);
            np += Bn.np;
            maxfn = mx;
            b2++;
        }
        DevBatch S{};
        S.pt0 = B0.pt0;
        S.np = np;
        S.sys = B0.sys;
        S.act0 = (int)t.sact.size();
        S.n_act = (int)uni.size();
        int fl = 0;
        for (int a : uni) {
            t.sact.push_back(DevAct{a, fl});
            fl += in.atom_nfn[a];
        }
        S.nfn = fl;
        t.sb.push_back(S);
        b = b2;
    }
    t.sb_first.push_back(in.n_batch);
}

int tc_build(TcPlan &t, const TcPlanInput &in, std::string *err)
{
    tc_free(t);
    build_super_batches(t, in, std::min(in.sb_points, kMaxBatchPoints), std::max(1.0, in.sb_growth));
    const int n_sb = (int)t.sb.size();
    t.batches.assign(n_sb, TcBatch{});
    t.sb_rank.assign(n_sb, -1);
    t.items.clear();
    t.waves.clear();
    size_t cap = (size_t)24 << 30;   // workloads up to ~24 GB of operand images run as one wave
    if (in.wave_mb > 0) cap = (size_t)in.wave_mb << 20;
    if (const char *e = getenv("FGI_TC_WAVE_MB")) cap = (size_t)std::max(1L, atol(e)) << 20;
    t.wave_cap = cap;
    // per-batch image geometry and footprint (3 planes always reserved)
    std::vector<size_t> foot(n_sb, 0);
    for (int b = 0; b < n_sb; b++) {
        const DevBatch &B = t.sb[b];
        TcBatch &T = t.batches[b];
        T.nrb = (B.nfn + 127) / 128;
        T.nc = (B.np + 63) / 64;
        T.nc_alloc = (T.nc + 1) / 2 * 2;
        T.nkc = (B.nfn + 63) / 64;
        T.plane_phi = (long long)T.nrb * T.nc_alloc * kChunkBytes;
        T.plane_d = (long long)T.nrb * T.nkc * kChunkBytes;
        foot[b] = 3 * (size_t)T.plane_phi + 3 * (size_t)std::max(T.plane_phi, T.plane_d);
        T.img_e = -1;
        if (in.with_e) foot[b] += 2 * (size_t)T.plane_phi;     // E in FP32: twice a BF16 plane
    }
    t.bound_grids = in.bound_grids;
    size_t max_ws = 0;
    TcWave w;
    size_t off = 0;
    auto close_wave = [&](int b_end) {
        w.nb = b_end - w.b0;
        if (w.nb <= 0) return;
        max_ws = std::max(max_ws, off);
        t.waves.push_back(w);
    };
    // each wave: the batches' images, then their partial densities (one row
    // of 128 doubles per (point tile, function block))
    long long part = 0;
    auto part_rows = [&](int b) { return (long long)(t.batches[b].nc_alloc / 2) * t.batches[b].nrb; };
    auto finish_wave = [&](int b_end) {
        w.part_off = (off + 1023) / 1024 * 1024;
        off = w.part_off + (size_t)part * 128 * sizeof(double);
        close_wave(b_end);
    };
    for (int b = 0; b < n_sb; b++) {
        const size_t pb = (size_t)part_rows(b) * 128 * sizeof(double);
        if (b > w.b0 && off + foot[b] + pb + (size_t)part * 1024 + 1024 > cap) {
            finish_wave(b);
            w = TcWave{};
            w.b0 = b;
            off = 0;
            part = 0;
        }
        TcBatch &T = t.batches[b];
        T.img_phi = (long long)off;
        T.img_aux = (long long)(off + 3 * (size_t)T.plane_phi);
        if (in.with_e) T.img_e = (long long)(off + 3 * (size_t)T.plane_phi + 3 * (size_t)std::max(T.plane_phi, T.plane_d));
        T.part0 = part;
        part += part_rows(b);
        off += foot[b];
    }
    finish_wave(n_sb);
    {
        size_t n_items = 0;   // the six lists below, for one allocation
        for (int b = 0; b < n_sb; b++) {
            if (t.sb[b].np <= 0 || t.sb[b].nfn <= 0) continue;
            const size_t nrb = (size_t)t.batches[b].nrb, nca = (size_t)t.batches[b].nc_alloc;
            n_items += 2 * nrb + nrb * (nrb + 1) / 2 + nca + nca / 2 + nrb * (nca / 2);
        }
        t.items.reserve(n_items);
    }
    for (TcWave &wv : t.waves) {
        // longest first: the wave's batches by contraction cost P n^2, each
        // batch's items kept together (they share image tiles in L2); the
        // persistent kernels stride over this list, so the small items land last
        std::vector<int> ord;
        for (int b = wv.b0; b < wv.b0 + wv.nb; b++)
            if (t.sb[b].np > 0 && t.sb[b].nfn > 0) ord.push_back(b);
        auto cost = [&](int b) { return (double)t.sb[b].np * t.sb[b].nfn * t.sb[b].nfn; };
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost(a) > cost(b); });
        for (size_t r = 0; r < ord.size(); r++) t.sb_rank[ord[r]] = (int)r;
        wv.phi0 = (long long)t.items.size();
        for (int b : ord)
            for (int I = 0; I < t.batches[b].nrb; I++) t.items.push_back(WorkItem{b, (short)I, 0});
        wv.nphi = (long long)t.items.size() - wv.phi0;
        wv.h0 = (long long)t.items.size();
        for (int b : ord)
            for (int I = 0; I < t.batches[b].nrb; I++)
                for (int J = I; J < t.batches[b].nrb; J++) t.items.push_back(WorkItem{b, (short)I, (short)J});
        wv.nh = (long long)t.items.size() - wv.h0;
        wv.g0 = (long long)t.items.size();
        for (int b : ord)
            for (int J = 0; J < t.batches[b].nrb; J++) t.items.push_back(WorkItem{b, (short)J, 0});
        wv.ng = (long long)t.items.size() - wv.g0;
        wv.pc0 = (long long)t.items.size();
        for (int b : ord)
            for (int c = 0; c < t.batches[b].nc_alloc; c++) t.items.push_back(WorkItem{b, (short)c, 0});
        wv.npc = (long long)t.items.size() - wv.pc0;
        wv.d0 = (long long)t.items.size();
        for (int b : ord)
            for (int mt = 0; mt < t.batches[b].nc_alloc / 2; mt++) t.items.push_back(WorkItem{b, (short)mt, 0});
        wv.nd = (long long)t.items.size() - wv.d0;
        // MMA items: J ascending (the longest contractions first), every point tile
        wv.e0 = (long long)t.items.size();
        for (int b : ord)
            for (int J = 0; J < t.batches[b].nrb; J++)
                for (int mt = 0; mt < t.batches[b].nc_alloc / 2; mt++)
                    t.items.push_back(WorkItem{b, (short)mt, (short)J});
        wv.ne = (long long)t.items.size() - wv.e0;
        for (int b = wv.b0; b < wv.b0 + wv.nb; b++) {
            const double P = t.sb[b].np, n = t.sb[b].nfn;
            wv.phi_flops += 30.0 * P * n;
            wv.phi_bytes += 32.0 * P + 12.0 * P * n;
            wv.h_flops += P * n * (n + 1.0);
            wv.h_bytes += 16.0 * n * (n + 1) / 2 + 12.0 * P * n;
            // symmetric D: the upper block triangle (about half of n^2)
            wv.n_flops += P * n * (n + 1.0) + 2.0 * P * n;
            wv.n_bytes += 3.0 * n * n + 6.0 * P * n + 16.0 * P;
            wv.g_bytes += 7.0 * n * n;
        }
    }
    // scratch before the images: the fixed-point H accumulator, or the
    // double-float copy of D followed by the per-function bounds of D
    t.nnz = in.nnz;
    t.n_fn = in.n_fn;
    t.bound_off = ((size_t)in.nnz * 8 + 255) / 256 * 256;
    t.sign_off = (t.bound_off + 8 * (size_t)in.n_fn + 255) / 256 * 256;
    t.img_base = (t.sign_off + 4 * (size_t)n_sb + 1023) / 1024 * 1024;
    t.ws_bytes = t.img_base + max_ws + 1024;
    // items must not be empty for the device copy
    if (!in.host_only) {
        const size_t nb_bytes = t.batches.size() * sizeof(TcBatch);
        const size_t ni_bytes = t.items.size() * sizeof(WorkItem);
        const size_t sb_bytes = t.sb.size() * sizeof(DevBatch);
        const size_t sa_bytes = t.sact.size() * sizeof(DevAct);
        auto al = [](size_t x) { return (x + 255) / 256 * 256; };
        const size_t tot = al(nb_bytes) + al(ni_bytes) + al(sb_bytes) + al(sa_bytes) + 256;
        cudaError_t e = cudaMalloc(&t.d_mem, tot);
        if (e != cudaSuccess) {
            t.d_mem = nullptr;
            *err = std::string("tensor-core plan: cudaMalloc failed: ") + cudaGetErrorString(e);
            return FGI_ERR_NOMEM;
        }
        char *base = (char *)t.d_mem;
        if (nb_bytes) cudaMemcpy(base, t.batches.data(), nb_bytes, cudaMemcpyHostToDevice);
        const size_t ioff = ((nb_bytes + 255) / 256) * 256;
        if (ni_bytes) cudaMemcpy(base + ioff, t.items.data(), ni_bytes, cudaMemcpyHostToDevice);
        t.d_batches = (const TcBatch *)base;
        t.d_items = (const WorkItem *)(base + ioff);
        const size_t soff = ioff + al(ni_bytes), aoff = soff + al(sb_bytes);
        if (sb_bytes) cudaMemcpy(base + soff, t.sb.data(), sb_bytes, cudaMemcpyHostToDevice);
        if (sa_bytes) cudaMemcpy(base + aoff, t.sact.data(), sa_bytes, cudaMemcpyHostToDevice);
        t.d_sb = (const DevBatch *)(base + soff);
        t.d_sact = (const DevAct *)(base + aoff);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&t.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (t.num_sms <= 0) t.num_sms = 1;
        e = set_attrs();
        if (e != cudaSuccess) {
            *err = std::string("tensor-core plan: cudaFuncSetAttribute: ") + cudaGetErrorString(e);
            return FGI_ERR_CUDA;
        }
    }
    t.built = true;
    return FGI_OK;
}

void tc_free(TcPlan &t)
{
    if (t.d_mem) cudaFree(t.d_mem);
    t.d_mem = nullptr;
    t.d_batches = nullptr;
    t.d_items = nullptr;
    t.built = false;
}

size_t tc_workspace_bytes(const TcPlan &t) { return t.ws_bytes; }

cudaError_t tc_launch_phi(const TcPlan &t, const DevPlan &P, const TcWave &w, const double *v, void *ws,
                          int n_split, cudaStream_t s)
{
    if (w.nphi <= 0) return cudaSuccess;
    // the H images (v given) of the split mode use the fixed-point leading term
    const int fixed = (v != nullptr && n_split == 3) ? 1 : 0;
    // the dynamic buffer caches geometry for the FP32 pass over the points
    // (bound_grids 0 and 1), or the point-atom distances of the table-bound pass
    const size_t dyn = smem_phi();
    k_tc_phi<<<(unsigned)w.nphi, kPhiThreads, dyn, s>>>(P, t.d_batches, t.d_items + w.phi0,
                                                       (uint8_t *)ws + t.img_base, v, n_split, fixed,
                                                       reinterpret_cast<int *>((uint8_t *)ws + t.sign_off),
                                                       t.bound_grids >= 2 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t tc_launch_phi_cols(const TcPlan &t, const DevPlan &P, const TcWave &w, void *ws, int n_split,
                               cudaStream_t s)
{
    if (w.npc <= 0) return cudaSuccess;
    k_tc_phi_cols<<<(unsigned)w.npc, kPhiThreads, 0, s>>>(P, t.d_batches, t.d_items + w.pc0,
                                                           (uint8_t *)ws + t.img_base, n_split,
                                                           t.bound_grids >= 1 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t tc_launch_h(const TcPlan &t, const DevPlan &P, const TcWave &w, const void *ws, int n_split,
                        cudaStream_t s)
{
    if (w.nh <= 0) return cudaSuccess;
    const int grid = (int)std::min<long long>(w.nh, t.num_sms);
    k_tc_h<<<grid, kThreadsTc, smem_tc_h(), s>>>(P, t.d_batches, t.d_items + w.h0, (int)w.nh,
                                                (const uint8_t *)ws + t.img_base, (unsigned long long *)ws, n_split,
                                                reinterpret_cast<const int *>((const uint8_t *)ws + t.sign_off));
    return cudaGetLastError();
}

cudaError_t tc_launch_fix_to_h(const TcPlan &t, const void *ws, double *h, long long nnz, int accumulate,
                               cudaStream_t s)
{
    (void)t;
    if (nnz <= 0) return cudaSuccess;
    k_fix_to_h<<<1216, 256, 0, s>>>((const long long *)ws, h, nnz, accumulate);
    return cudaGetLastError();
}

cudaError_t tc_launch_gather_d(const TcPlan &t, const DevPlan &P, const TcWave &w, double offdiag_scale,
                               void *ws, int n_split, cudaStream_t s, bool full)
{
    if (w.ng <= 0) return cudaSuccess;
    const char *base = (const char *)ws;
    k_tc_gather_d<<<(unsigned)w.ng, 256, 0, s>>>(P, t.d_batches, t.d_items + w.g0, (uint8_t *)ws + t.img_base,
                                                 (const float2 *)base, (const unsigned int *)(base + t.bound_off),
                                                 (const float *)(base + t.bound_off + 4 * t.n_fn),
                                                 (float)offdiag_scale, n_split, full ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t tc_launch_to_df(const TcPlan &t, const DevPlan &P, const double *x, void *ws, const long long *sys_val0,
                            const long long *sys_nnz, const int *fn_sys, cudaStream_t s)
{
    if (t.nnz <= 0) return cudaSuccess;
    char *base = (char *)ws;
    unsigned int *gmax = (unsigned int *)(base + t.bound_off);
    float *gsum = (float *)(base + t.bound_off + 4 * t.n_fn);
    cudaError_t e = cudaMemsetAsync(gmax, 0, 8 * (size_t)t.n_fn, s);
    if (e != cudaSuccess) return e;
    k_to_df<<<1216, 256, 0, s>>>(x, (float2 *)base, P.rowptr, fn_sys, sys_val0, sys_nnz, t.n_fn, gmax, gsum);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_d_colbounds<<<1216, 256, 0, s>>>((const float2 *)base, P.col_glob, t.nnz, gmax, gsum);
    return cudaGetLastError();
}

cudaError_t tc_launch_density(const TcPlan &t, const DevPlan &P, const TcWave &w, const void *ws, double *n,
                              int n_split, cudaStream_t s)
{
    if (w.nd <= 0) return cudaSuccess;
    double *part = reinterpret_cast<double *>((uint8_t *)const_cast<void *>(ws) + t.img_base + w.part_off);
    const int grid = (int)std::min<long long>(w.ne, t.num_sms);
    k_tc_density<false><<<grid, kThreadsTc, smem_tc(3), s>>>(P, t.d_batches, t.d_items + w.e0, (int)w.ne,
                                                             (const uint8_t *)ws + t.img_base, part, n_split,
                                                             nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_density_sum<<<(unsigned)w.nd, 128, 0, s>>>(P, t.d_batches, t.d_items + w.d0, part, n, 2.0);
    return cudaGetLastError();
}

cudaError_t tc_launch_adjoint(const TcPlan &t, const DevPlan &P, const TcWave &w, const void *ws, const double *v,
                              double *dv, double *dR, int n_split, cudaStream_t s)
{
    if (w.nd <= 0) return cudaSuccess;
    if (!t.batches.empty() && t.batches[w.b0].img_e < 0) return cudaErrorInvalidValue;   // no room for E
    uint8_t *img = (uint8_t *)const_cast<void *>(ws) + t.img_base;
    double *part = reinterpret_cast<double *>(img + w.part_off);
    const int grid = (int)std::min<long long>(w.ne, t.num_sms);
    k_tc_density<true><<<grid, kThreadsTc, smem_tc(3), s>>>(P, t.d_batches, t.d_items + w.e0, (int)w.ne, img, part,
                                                            n_split, img);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_density_sum<<<(unsigned)w.nd, 128, 0, s>>>(P, t.d_batches, t.d_items + w.d0, part, dv, 1.0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tc_adj_grad<<<(unsigned)w.npc, 256, 0, s>>>(P, t.d_batches, t.d_items + w.pc0, img, v, dR);
    return cudaGetLastError();
}

// Self-test of the failure path: one CTA waits on an mbarrier that nothing
// completes.  The bounded wait gives up after kWaitLimitNs and records the
// time-out in the status word, as a stalled pipeline would; no fault, no hang.
__global__ void k_wait_selftest(int *status)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_a(&bar, 0, status, &abort_flag);
}

cudaError_t tc_launch_wait_selftest(int *status, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(status);
    return cudaGetLastError();
}

}  // namespace fgi
