// gf_dfloat.cuh -- double-float arithmetic (an unevaluated sum hi + lo of two
// floats, ~48-bit significand) and the double-float Gaussian-blob evaluator
// of the GF_F64X mode.
//
// On GB300 the FP64 pipe retires 2 lanes per clock per SM against 128 for
// FP32, so the blob terms -- about 80% of the FP64 instructions of a GRIN ray step --
// are computed here with error-free transformations on the FP32 pipe and only
// their sums are returned in double:
//   two_sum (Knuth, TAOCP vol. 2), fast_two_sum and two_prod via FMA
//   (Dekker 1971), and the double-word algorithms of Joldes, Muller & Popescu,
//   "Tight and rigorous error bounds for basic building blocks of double-word
//   arithmetic", ACM TOMS 44 (2017): AccurateDWPlusDW (relative error
//   <= 3u^2 + 13u^3), SloppyDWPlusDW (where no cancellation matters),
//   DWTimesDW2 (<= 5u^2), DWTimesFP2, u = 2^-24.
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

// The conversions between double and float run on the FP64 pipe, which the
// rest of the ray step keeps busy; these do them on the bit patterns with
// integer operations instead.

// x rounded to the nearest float (ties to even, as the hardware conversion)
// for 2^-126 <= |x| < 2^128 - 2^103; smaller |x| gives a zero of x's sign,
// larger |x|, inf and NaN give inf.
__device__ __forceinline__ float narrow_rn(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned mag = hi & 0x7fffffffu;
    unsigned f = ((mag - ((1023u - 127u) << 20)) << 3) | (lo >> 29);
    const unsigned drop = lo & 0x1fffffffu;   // the 29 bits below the float's last place
    f += (drop > 0x10000000u || (drop == 0x10000000u && (f & 1u))) ? 1u : 0u;   // carries into the exponent
    f = mag < ((1023u - 126u) << 20) ? 0u : (mag >= ((1023u + 128u) << 20) ? 0x7f800000u : f);
    return __uint_as_float((hi & 0x80000000u) | f);
}

// double -> (hi, lo): hi = x rounded to float, lo = the exact remainder
// x - hi rounded to float (one FP64 subtraction); ~2^-48 relative for
// 2^-126 <= |x| < 2^128 (positions and directions of rays).
__device__ __forceinline__ dfl df_from_double(double x)
{
    const float hi = narrow_rn(x);
    return {hi, narrow_rn(x - widen(hi))};
}

__device__ __forceinline__ double df_to_double(dfl x) { return widen(x.hi) + widen(x.lo); }

// 2^a for -63 < a <= 0 in double-float: Tang's table-driven method in base
// 2 with a 2048-entry table, so that the reduction is exact.  k =
// round(2048 a.hi) (adding 1.5 * 2^23 rounds 2048 a.hi to an integer), rh =
// a.hi - k/2048 exact with |rh| <= 2^-12, r = rh + a.lo; then
// 2^r - 1 = c1 r + c2 r^2 + c3 r^3 (truncation below (r ln2)^4/24 < 4e-17):
// c1 rh in double-float, the small rest c1 a.lo + c2 r^2 + c3 r^3 (below
// 3.5e-8 for |a| <= 1) in float; the result T (1 + p) with T = 2^(j/2048) a
// float pair, summed with error-free transformations and renormalised, times
// 2^(k >> 11).  Relative error about 2^-47 max(1, |a|) (a.lo enters through
// one float product), median ~2^-50.  sT: the (hi, lo) table in shared memory.
// Table entries 2^(j/2048) as float pairs: from the double-float table, or
// split from the FP64 table (hi = RN_float(T_j), lo = RN_float(T_j - hi):
// one FP64 subtraction, 48 of its 53 bits).
struct DfTabPairs {
    const float *__restrict__ sT;
    __device__ __forceinline__ dfl operator()(int j) const { return {sT[2 * j], sT[2 * j + 1]}; }
};
struct DfTabFromDouble {
    const double *__restrict__ T;
    __device__ __forceinline__ dfl operator()(int j) const { return df_from_double(T[j]); }
};

template <typename Tab>
__device__ __forceinline__ dfl df_exp2_tab(dfl a, const Tab &tab)
{
    const float tf = __fmaf_rn(a.hi, 2048.0f, 12582912.0f);           // 1.5 * 2^23 + k
    const int k = __float_as_int(tf) - 0x4B400000;                      // bits of 1.5 * 2^23
    const float kf = __fsub_rn(tf, 12582912.0f);                        // exact
    const float rh = __fmaf_rn(kf, -0x1p-11f, a.hi);                    // exact
    const float rs = __fadd_rn(rh, a.lo);
    const dfl P1 = df_mul_f(dfl{kDfC1Hi, kDfC1Lo}, rh);
    const float small = __fmaf_rn(__fmul_rn(rs, rs), __fmaf_rn(rs, kDfC3, kDfC2), __fmul_rn(kDfC1Hi, a.lo));
    const float plo = __fadd_rn(P1.lo, small);                          // p = P1.hi + plo
    const int j = k & (kDfExpN - 1);
    const dfl T = tab(j);
    // T (1 + p) = T.hi + T.hi P1.hi + [T.lo + (T.lo P1.hi + T.hi plo + error of T.hi P1.hi)]
    const dfl ph = two_prod(T.hi, P1.hi);
    const float tl = __fmaf_rn(T.lo, P1.hi, __fmaf_rn(T.hi, plo, ph.lo));
    const dfl s = fast_two_sum(T.hi, ph.hi);
    const dfl u = two_sum(s.lo, T.lo);
    const dfl v = fast_two_sum(s.hi, u.hi);
    const dfl G = fast_two_sum(v.hi, __fadd_rn(v.lo, __fadd_rn(tl, u.lo)));
    const float sc = __int_as_float((127 + (k >> 11)) << 23);           // 2^(k >> 11), k >> 11 >= -64
    return {__fmul_rn(G.hi, sc), __fmul_rn(G.lo, sc)};
}

__device__ __forceinline__ dfl df_exp2(dfl a, const float *__restrict__ sT)
{
    return df_exp2_tab(a, DfTabPairs{sT});
}

static __constant__ float c_dfexp2_tab[2 * kDfExpN] = {GF_DFEXP2_TAB_VALUES};

__device__ __forceinline__ void stage_dfexp_table(float *sT)
{
    for (int j = threadIdx.x; j < 2 * kDfExpN; j += blockDim.x) sT[j] = c_dfexp2_tab[j];
}

// Double-float blob row: c_hi[3], c_lo[3], then the pairs of s2 = s/ln2 (the
// exponent in base 2), A and B = 2 s A, each value split exactly as
// hi = RN_float(v), lo = RN_float(v - hi).  Built on the host with the medium.
constexpr int kDfBlobStride = kDfRowFloats;

__device__ __forceinline__ void stage_df_blobs(const MediumParams &m, float *sd)
{
    for (int j = threadIdx.x; j < m.n_blobs * kDfBlobStride; j += blockDim.x) sd[j] = m.dfrows[j];
}

// Sum over blobs of A_j exp(s_j |x - c_j|^2) and of its gradient, in
// double-float, added to n2 and g in double.  Field f of blob j is read from
// sd[(kDfBlobStride j + f) * stride] (stride 1: a block-shared table; stride
// = lanes: one table per lane).  Terms whose base-2 exponent s2 |x - c|^2 is
// below -58.5 are skipped (as in the FP64 evaluator); a float pre-test with
// a margin of 1 (kDfPreCull2) removes most of them before any double-float work.
constexpr float kDfPreCull2 = 59.5f;

__device__ __forceinline__ void blobs_df(const float *__restrict__ sd, int nb, const double *x, double &n2,
                                         double *g, const float *__restrict__ sT, int &live, int stride = 1)
{
    const dfl X0 = df_from_double(x[0]), X1 = df_from_double(x[1]), X2 = df_from_double(x[2]);
    dfl N = {0.f, 0.f}, G0 = {0.f, 0.f}, G1 = {0.f, 0.f}, G2 = {0.f, 0.f};
    for (int j = 0; j < nb; ++j) {
        const float *bp = sd + kDfBlobStride * j * stride;
        const auto b = [&](int f) { return bp[f * stride]; };   // read where used
        const float ex = X0.hi - b(0), ey = X1.hi - b(1), ez = X2.hi - b(2);
        if ((ex * ex + ey * ey + ez * ez) * b(6) < -kDfPreCull2) continue;
        const dfl d0 = df_add(X0, dfl{-b(0), -b(3)});
        const dfl d1 = df_add(X1, dfl{-b(1), -b(4)});
        const dfl d2 = df_add(X2, dfl{-b(2), -b(5)});
        const dfl q = df_add_sloppy(df_add_sloppy(df_sqr(d0), df_sqr(d1)), df_sqr(d2));   // no cancellation
        const dfl a = df_mul(dfl{b(6), b(7)}, q);
        if (a.hi < (float)kBlobCull2) continue;
        const dfl E = df_exp2(a, sT);
        const dfl AG = df_mul(dfl{b(8), b(9)}, E);
        N = df_add_sloppy(N, AG);                                    // absolute error ~u^2 |N|, |AG|
        const dfl c = df_mul(dfl{b(10), b(11)}, E);                 // 2 s A G
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
    return rhs_iso_from_index<double, WANT_D>(om, y, n2, g, f, D);
}

}  // namespace gf
