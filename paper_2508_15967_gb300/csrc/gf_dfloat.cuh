// gf_dfloat.cuh -- double-float arithmetic (an unevaluated sum hi + lo of two
// floats, ~48-bit significand) and the double-float Gaussian-blob evaluator
// of the GF_F64X mode.
//
// On GB300 the FP64 pipe retires 2 lanes per clock per SM against 128 for
// FP32, so the blob terms -- 86% of the FP64 instructions of a GRIN ray step --
// are computed here with error-free transformations on the FP32 pipe and only
// their sums are returned in double:
//   two_sum (Knuth, TAOCP vol. 2), fast_two_sum and two_prod via FMA
//   (Dekker 1971), and the double-word algorithms of Joldes, Muller & Popescu,
//   "Tight and rigorous error bounds for basic building blocks of double-word
//   arithmetic", ACM TOMS 44 (2017): AccurateDWPlusDW (relative error
//   <= 3u^2 + 13u^3), SloppyDWPlusDW (where no cancellation matters),
//   DWPlusFP, DWTimesDW2 (<= 5u^2), DWTimesFP2, u = 2^-24.
// Every operation uses explicitly rounded intrinsics so that the compiler
// neither contracts nor reassociates them.
#pragma once

#include "gf_internal.cuh"

namespace gf {

#include "gf_dfexp_table.inc"

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, err};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ dfl fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// AccurateDWPlusDW
__device__ __forceinline__ dfl df_add(dfl x, dfl y)
{
    const dfl s = two_sum(x.hi, y.hi);
    const dfl t = two_sum(x.lo, y.lo);
    const dfl v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

// SloppyDWPlusDW: 11 operations against 20; no relative error bound when x
// and y nearly cancel, but |error| <= ~2 u^2 (|x| + |y|) always, so it serves
// sums whose absolute error is what matters (sums of squares, accumulations
// into a running total of larger magnitude).
__device__ __forceinline__ dfl df_add_sloppy(dfl x, dfl y)
{
    const dfl s = two_sum(x.hi, y.hi);
    const float v = __fadd_rn(x.lo, y.lo);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, v));
}

// DWPlusFP
__device__ __forceinline__ dfl df_add_f(dfl x, float y)
{
    const dfl s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}

// DWTimesDW2
__device__ __forceinline__ dfl df_mul(dfl x, dfl y)
{
    const dfl c = two_prod(x.hi, y.hi);
    const float tl = __fmaf_rn(x.lo, y.hi, __fmul_rn(x.hi, y.lo));
    return fast_two_sum(c.hi, __fadd_rn(c.lo, tl));
}

// DWTimesFP2
__device__ __forceinline__ dfl df_mul_f(dfl x, float y)
{
    const dfl c = two_prod(x.hi, y);
    return fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}

__device__ __forceinline__ dfl df_sqr(dfl x)
{
    const float p = __fmul_rn(x.hi, x.hi);
    float e = __fmaf_rn(x.hi, x.hi, -p);
    e = __fmaf_rn(__fmul_rn(2.0f, x.hi), x.lo, e);
    return fast_two_sum(p, e);
}

// exact double -> (hi, lo) split; the remainder x - hi is exact in double
__device__ __forceinline__ dfl df_from_double(double x)
{
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ double df_to_double(dfl x) { return (double)x.hi + (double)x.lo; }

// exp(a) for -44 < a <= 0 in double-float: Tang's table-driven method with
// k = round(64 a / ln2), r = a - k ln2/64 (ln2/64 = L1 + L2 + L3 + L4 with
// k Li exact for i <= 3), expm1(r) = r + r^2/2 + r^3/6 + r^4 (1/24 + r/120)
// (the last group in float is enough: r^4/24 < 4e-11), result
// 2^(k >> 6) (T_j + T_j expm1(r)) with T_j = 2^(j/64) as a float pair.
// sT: the 128-float (hi, lo) table in shared memory.
__device__ __forceinline__ dfl df_exp(dfl a, const float *__restrict__ sT)
{
    const float kf = rintf(__fmul_rn(a.hi, kDfInvL));
    const float t1 = __fmaf_rn(-kf, kDfL1, a.hi);                 // exact
    dfl r = two_sum(t1, __fmul_rn(-kf, kDfL2));                   // exact product
    r = df_add_f(r, a.lo);
    r = df_add_f(r, __fmul_rn(-kf, kDfL3));                       // exact product
    r = fast_two_sum(r.hi, __fmaf_rn(-kf, kDfL4, r.lo));
    const dfl r2 = df_sqr(r);
    const dfl r3 = df_mul(r2, r);
    // no cancellation in the polynomial (|r^2/2| < 3e-3 |r|) or in T + T p
    // (|p| < 6e-3): the sloppy double-word sum keeps its 2 u^2 error there
    dfl p = df_add_sloppy(r, dfl{__fmul_rn(0.5f, r2.hi), __fmul_rn(0.5f, r2.lo)});
    p = df_add_sloppy(p, df_mul(r3, dfl{kDfSixthHi, kDfSixthLo}));
    const float r4 = __fmul_rn(r2.hi, r2.hi);
    p = df_add_f(p, __fmul_rn(r4, __fmaf_rn(r.hi, 1.0f / 120.0f, 1.0f / 24.0f)));
    const int k = (int)kf;
    const int j = k & 63;
    const dfl T = {sT[2 * j], sT[2 * j + 1]};
    const dfl G = df_add_sloppy(T, df_mul(T, p));
    const float sc = __int_as_float((127 + (k >> 6)) << 23);      // 2^(k >> 6), k >> 6 >= -64
    return {__fmul_rn(G.hi, sc), __fmul_rn(G.lo, sc)};
}

static __constant__ float c_dfexp2_tab[128] = {
#define GF_T8(i) kDfExp2Tab[i], kDfExp2Tab[i + 1], kDfExp2Tab[i + 2], kDfExp2Tab[i + 3], \
                 kDfExp2Tab[i + 4], kDfExp2Tab[i + 5], kDfExp2Tab[i + 6], kDfExp2Tab[i + 7]
    GF_T8(0),  GF_T8(8),  GF_T8(16), GF_T8(24), GF_T8(32), GF_T8(40), GF_T8(48), GF_T8(56),
    GF_T8(64), GF_T8(72), GF_T8(80), GF_T8(88), GF_T8(96), GF_T8(104), GF_T8(112), GF_T8(120)
#undef GF_T8
};

__device__ __forceinline__ void stage_dfexp_table(float *sT)
{
    for (int j = threadIdx.x; j < 128; j += blockDim.x) sT[j] = c_dfexp2_tab[j];
}

// Double-float blob row: c_hi[3], c_lo[3], s_hi, s_lo, A_hi, A_lo, each
// value split exactly as hi = RN_float(v), lo = RN_float(v - hi) (2 s is
// formed exactly by doubling s).  Built on the host with the medium.
constexpr int kDfBlobStride = kDfRowFloats;

__device__ __forceinline__ void stage_df_blobs(const MediumParams &m, float *sd)
{
    for (int j = threadIdx.x; j < m.n_blobs * kDfBlobStride; j += blockDim.x) sd[j] = m.dfrows[j];
}

// Sum over blobs of A_j exp(s_j |x - c_j|^2) and of its gradient, in
// double-float, added to n2 and g in double.  Field f of blob j is read from
// sd[(kDfBlobStride j + f) * stride] (stride 1: a block-shared table; stride
// = lanes: one table per lane).  Terms whose exponent is below -40.5 are
// skipped (as in the FP64 evaluator); a float pre-test with margin removes
// most of them before any double-float work.
__device__ __forceinline__ void blobs_df(const float *__restrict__ sd, int nb, const double *x, double &n2,
                                         double *g, const float *__restrict__ sT, int &live, int stride = 1)
{
    const dfl X0 = df_from_double(x[0]), X1 = df_from_double(x[1]), X2 = df_from_double(x[2]);
    dfl N = {0.f, 0.f}, G0 = {0.f, 0.f}, G1 = {0.f, 0.f}, G2 = {0.f, 0.f};
    for (int j = 0; j < nb; ++j) {
        const float *bp = sd + kDfBlobStride * j * stride;
        const auto b = [&](int f) { return bp[f * stride]; };   // read where used
        const float ex = X0.hi - b(0), ey = X1.hi - b(1), ez = X2.hi - b(2);
        if ((ex * ex + ey * ey + ez * ez) * b(6) < -kBlobCullQF) continue;
        const dfl d0 = df_add(X0, dfl{-b(0), -b(3)});
        const dfl d1 = df_add(X1, dfl{-b(1), -b(4)});
        const dfl d2 = df_add(X2, dfl{-b(2), -b(5)});
        const dfl q = df_add_sloppy(df_add_sloppy(df_sqr(d0), df_sqr(d1)), df_sqr(d2));   // no cancellation
        const dfl s = {b(6), b(7)};
        const dfl a = df_mul(s, q);
        if (a.hi < (float)kBlobCull) continue;
        const dfl AG = df_mul(dfl{b(8), b(9)}, df_exp(a, sT));
        N = df_add_sloppy(N, AG);                                    // absolute error ~u^2 |N|, |AG|
        const dfl c = df_mul(dfl{2.f * s.hi, 2.f * s.lo}, AG);      // 2 s A G
        G0 = df_add_sloppy(G0, df_mul(c, d0));
        G1 = df_add_sloppy(G1, df_mul(c, d1));
        G2 = df_add_sloppy(G2, df_mul(c, d2));
        ++live;
    }
    n2 += df_to_double(N);
    g[0] += df_to_double(G0);
    g[1] += df_to_double(G1);
    g[2] += df_to_double(G2);
}

// Ray right-hand side of an isotropic medium with the blob sums in
// double-float (GF_F64X): base index law, D and f in FP64 exactly as
// rhs_iso, blob terms from blobs_df over the rows in sd (stride as there).
template <int KIND, bool WANT_D>
__device__ __forceinline__ bool rhs_df(const MediumParams &m, const float *__restrict__ sd, int nb, int stride,
                                       const Omega<double> &om, const double *y, double *f, double &D,
                                       const float *__restrict__ dT, int &live)
{
    double n2, g[3];
    EvalCtx<double> base;
    iso_index<double, KIND>(m, nullptr, 0, y, n2, g, base);
    blobs_df(sd, nb, y, n2, g, dT, live, stride);
    if constexpr (WANT_D) D = y[3] * y[3] + y[4] * y[4] + y[5] * y[5] - om.w * om.w * n2;
    if (!(n2 > 0.0)) return false;
    const double inv = 1.0 / n2;
    const double a = inv * om.inv_w, b = om.half_w * inv;
    f[0] = a * y[3];
    f[1] = a * y[4];
    f[2] = a * y[5];
    f[3] = b * g[0];
    f[4] = b * g[1];
    f[5] = b * g[2];
    return true;
}

}  // namespace gf
