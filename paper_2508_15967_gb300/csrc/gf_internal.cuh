// gf_internal.cuh -- internal declarations shared by the library's translation
// units: the device-side medium parameters, the fused D / grad D evaluators and
// host error helpers.  Not part of the public ABI (include/gf.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gf.h"

namespace gf {

enum : int { K_HOMOG = GF_MED_HOMOG, K_LUNEBURG = GF_MED_LUNEBURG, K_GRIN = GF_MED_GRIN,
             K_QUADRATIC = GF_MED_QUADRATIC, K_SPLINE = GF_MED_SPLINE, K_COLD = GF_MED_COLD };

// Device blob rows, 6 values each:
//   plain  (adjoint sweep, double-float path): A, cx, cy, cz, s = -1 / (2 w^2), 2 s
//   scaled (FP64 evaluator; a float copy for the FP32 evaluator):
//          sigma, -sigma cx, -sigma cy, -sigma cz, A, -2 ln2 sigma A
// with sigma = sqrt(-s / ln2), so that A exp(s |x - c|^2) = A 2^(-|u|^2),
// u = sigma x - sigma c, and grad (A 2^(-|u|^2)) = (-2 ln2 sigma A) 2^(-|u|^2) u.
constexpr int kBlobStride = 6;
constexpr double kInvLn2 = 0x1.71547652b82fep+0;    // 1/ln2, rounded
constexpr double kNeg2Ln2 = -0x1.62e42fefa39efp+0;  // -2 ln2, rounded
constexpr int kDfRowFloats = 12;   // double-float blob row (GF_F64X), see gf_dfloat.cuh

// Medium as the kernels see it (passed by value as a kernel argument).
struct MediumParams {
    int32_t kind, n_blobs, grid_n;
    float pre_lim;               // FP32 pre-test valid while max_i |x_i| <= pre_lim
    double n_h2;                 // homogeneous n^2
    double n02, n02a2;           // GRIN: n0^2 and n0^2 a^2
    const double *blobs64;       // n_blobs plain rows
    const float *blobs32;        // float copy of the scaled rows
    const double *blobs64s;      // n_blobs scaled rows
    const float *pre32;          // n_blobs x 4 floats: sigma, -sigma cx, -sigma cy, -sigma cz
    const float *dfrows;         // n_blobs double-float rows (GF_F64X; layout in gf_dfloat.cuh)
    const float4 *grid;          // grid_n^3 nodes x 2 float4
    int32_t n_species, pad2;     // cold plasma
    double species[2 * GF_MAX_SPECIES];   // (w_p^2, Omega) per species
    double prof[4];                       // f = prof0 + prof1 x_0, g = prof2 + prof3 x_0
    double cold_x[3 * GF_MAX_SPECIES];    // per species w_p^2 f', Omega g', 2 Omega g'
    double wp_sum;                        // sum of the species' w_p^2
};

// Ray buffers with a typed state pointer.
template <typename R>
struct RaysView {
    int64_t n, ld;
    R *y;
    double *t;
    int32_t *status, *steps;
    double *d_res, *d_max;
};

}  // namespace gf

// A device medium: parameters for the built-in kernels, or a generated RK4
// kernel compiled at run time (jit_lib != nullptr).
struct gf_medium_s {
    gf::MediumParams p{};
    int device = -1;
    double *d_blobs64 = nullptr;     // plain rows, then scaled rows (2 x n_blobs rows)
    float *d_blobs32 = nullptr;      // float scaled rows, pre-test rows, double-float rows
    float4 *d_grid = nullptr;
    cudaLibrary_t jit_lib = nullptr;
    cudaKernel_t jit_kernel = nullptr;
};

namespace gf {

// ------------------------------------------------------------------ host side

void set_error(const char *fmt, ...);
gf_status cuda_status(cudaError_t e, const char *what);
// Device allocations of the library (counted; see gf_bench_live_allocations).
cudaError_t dev_alloc(void **p, size_t bytes);
template <typename T>
inline cudaError_t dev_alloc(T **p, size_t bytes)
{
    return dev_alloc(reinterpret_cast<void **>(p), bytes);
}
void dev_free(void *p);   // NULL: no-op
gf_status check_rays(const gf_rays *r, bool need_state);
gf_status check_device_ptr(const void *p, const char *name);
const MediumParams &params_of(gf_medium m);
unsigned long long *work_counters();   // device counters set by gf_bench_set_counters, or NULL
int device_of(gf_medium m);

// Per-translation-unit launchers (return cudaGetLastError() of the launch).
cudaError_t launch_rk4(const MediumParams &m, gf_precision prec, const gf_rays &r, double omega,
                       double dt, int64_t n_steps, double radius, int64_t every, double *ckpt,
                       cudaStream_t s);
size_t adjoint_scratch_bytes(int nb, int64_t n, int64_t every);
cudaError_t launch_adjoint(const MediumParams &m, int64_t n, double omega, double dt, int64_t n_steps,
                           int64_t every, const double *ckpt, const int32_t *steps_done, const double *lambda,
                           int64_t ld, double *dtheta, double *dy0, void *scratch, cudaStream_t s);
cudaError_t launch_rk4_jit(gf_medium m, const gf_rays &r, double omega, double dt, int64_t n_steps,
                           double radius, cudaStream_t s);
cudaError_t launch_newton_kx(const MediumParams &m, gf_precision prec, const gf_rays &r, double omega, double tol,
                             int max_iter, cudaStream_t s);
cudaError_t launch_onshell(const MediumParams &m, gf_precision prec, const gf_rays &r,
                           const void *dir, double omega, cudaStream_t s);

// ---------------------------------------------------------------- device side

#include "gf_exp_table.inc"

constexpr int kExpTabN = 2048;

// 2^(j/2048), j = 0..2047 (one copy per translation unit in global memory,
// staged into shared memory by every block that evaluates blob terms in FP64).
static __device__ double g_exp2_tab[kExpTabN] = {GF_EXP2_TAB_VALUES};

__device__ __forceinline__ void stage_exp_table(double *sT)
{
    for (int j = threadIdx.x; j < kExpTabN; j += blockDim.x) sT[j] = g_exp2_tab[j];
}

// x rounded toward zero to float, on the bit pattern with integer operations
// (the FP64 pipe also executes the hardware conversion): exact sign, exponent
// and leading 23 fraction bits for 2^-126 <= |x| < 2^128 (relative error
// below 2^-23); smaller |x| gives 0, larger |x|, inf and NaN give inf.
__device__ __forceinline__ float narrow_trunc(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned mag = hi & 0x7fffffffu;
    unsigned f = ((mag - ((1023u - 127u) << 20)) << 3) | (lo >> 29);
    f = mag < ((1023u - 126u) << 20) ? 0u : (mag >= ((1023u + 128u) << 20) ? 0x7f800000u : f);
    return __uint_as_float((hi & 0x80000000u) | f);
}

// v as a double, on the bit pattern with integer operations (the hardware
// conversion runs on the FP64 pipe): exact for zeros, normal floats, inf and NaN; subnormal
// floats (below 1.2e-38) become a zero of their sign.
__device__ __forceinline__ double widen(float v)
{
    const unsigned b = __float_as_uint(v);
    const unsigned mag = b & 0x7fffffffu, sign = b & 0x80000000u;
    const unsigned adj = mag >= 0x7f800000u ? (2047u - 255u) << 20 : (1023u - 127u) << 20;
    const bool tiny = mag < 0x00800000u;
    return __hiloint2double((int)(tiny ? sign : sign | ((mag >> 3) + adj)), tiny ? 0 : (int)(b << 29));
}

// 1/v for v > 0: the FP32 reciprocal of v's leading 24 bits, widened on the
// bit pattern, is a seed r with relative error |d| < 2^-22; one Newton step
// of cubic order, r (1 + e + e^2) with e = 1 - v r, leaves |d|^3 < 2^-66
// before the final rounding (within one ulp of 1/v), in 3 FP64 operations.
// Outside 2^-120 <= v < 2^120 (or for inf, NaN) the IEEE division is used.
__device__ __forceinline__ double recip_pos(double v)
{
    const unsigned hi = (unsigned)__double2hiint(v);
    if (hi - ((1023u - 120u) << 20) >= (240u << 20)) return 1.0 / v;
    const float vf = __uint_as_float(((hi - ((1023u - 127u) << 20)) << 3) | ((unsigned)__double2loint(v) >> 29));
    const unsigned rb = __float_as_uint(__frcp_rn(vf));
    const double r = __hiloint2double((int)((rb >> 3) + ((1023u - 127u) << 20)), (int)(rb << 29));
    const double e = fma(-v, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// 1/v for v > 0 to a relative error below 2^-44: the same FP32 seed refined by
// one Newton step of quadratic order, r (1 + e), in 2 FP64 operations (for
// error measures, where a few ulps do not matter).  Outside 2^-120 <= v < 2^120
// the IEEE division.
__device__ __forceinline__ double recip_pos_q(double v)
{
    const unsigned hi = (unsigned)__double2hiint(v);
    if (hi - ((1023u - 120u) << 20) >= (240u << 20)) return 1.0 / v;
    const float vf = __uint_as_float(((hi - ((1023u - 127u) << 20)) << 3) | ((unsigned)__double2loint(v) >> 29));
    const unsigned rb = __float_as_uint(__frcp_rn(vf));
    const double r = __hiloint2double((int)((rb >> 3) + ((1023u - 127u) << 20)), (int)(rb << 29));
    return fma(r, fma(-v, r, 1.0), r);
}

// The bits of a double a below the 24 that narrow_trunc(a) keeps, as two
// floats with a's sign: a = narrow_trunc(a) + t1 + t2 exactly, t1 holding the
// next 23 significand bits and t2 the last 6, for 2^-74 <= |a| < 2^11.
// Smaller |a| give t1 = t2 = 0 (the bits dropped are below 2^-97).  Each part
// is a small integer turned into a float by the 2^23 bias trick and scaled by a
// power of two built on its bit pattern: integer and FP32 operations only.
__device__ __forceinline__ void tail_floats(double a, float &t1, float &t2)
{
    const unsigned hi = (unsigned)__double2hiint(a), lo = (unsigned)__double2loint(a);
    const unsigned eb = (hi >> 20) & 0x7FFu;                 // biased exponent E + 1023
    const unsigned sgn = hi & 0x80000000u;
    const float m1 = __fsub_rn(__uint_as_float(0x4B000000u | ((lo >> 6) & 0x7FFFFFu)), 8388608.0f);
    const float m2 = __fsub_rn(__uint_as_float(0x4B000000u | (lo & 0x3Fu)), 8388608.0f);
    const bool ok = eb - 949u < 85u;                          // 949 <= eb <= 1033
    const float s1 = __uint_as_float(sgn | ((eb - 942u) << 23));   // +-2^(E - 46)
    const float s2 = __uint_as_float(sgn | ((eb - 948u) << 23));   // +-2^(E - 52)
    t1 = ok ? __fmul_rn(m1, s1) : 0.0f;
    t2 = ok ? __fmul_rn(m2, s2) : 0.0f;
}

// x 2^63 truncated toward zero, as a signed 64-bit integer, for a float
// |x| < 2^-11 (its significand shifted into place; zero and subnormals give 0).
__device__ __forceinline__ long long fix63(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned long long m = (b & 0x7FFFFFu) | 0x800000u;
    const int sh = (int)e - 87;                                   // x = m 2^(e - 150)
    unsigned long long v = sh >= 0 ? m << min(sh, 63) : m >> min(-sh, 63);   // shifts kept below 64
    v = e == 0u ? 0ull : v;
    return (b >> 31) ? -(long long)v : (long long)v;
}

// x truncated toward zero to a multiple of 2^-63 (fix63(x) 2^-63 as a float:
// the fraction bits below 2^-63 cleared; zero and subnormals give 0).
__device__ __forceinline__ float trunc63(float x)
{
    const unsigned b = __float_as_uint(x);
    const int nclr = 87 - (int)((b >> 23) & 0xFFu);              // fraction bits below 2^-63
    const unsigned keep = nclr <= 0 ? 0xFFFFFFFFu : (nclr >= 24 ? 0u : ~((1u << nclr) - 1u));
    return __uint_as_float(b & keep);
}

// The reduction and polynomial of the blob exponential (exp2_tab_int,
// exp2_tab_fp), on the FP32 and integer pipes: k = round(2048 a) and
// e^t - 1 = ph + pl with t = (a - k/2048) ln2.
struct Exp2Red {
    int k;
    float ph, pl;
};

// e^t - 1 = ph + pl for t = r ln2, r = rh + rl given as a float pair
// (|r| <= 2^-12 + 2^-23 |a|, |rl| below 2^-34 or one ulp of rh).
__device__ __forceinline__ Exp2Red exp2_poly(int k, float rh, float rl)
{
    // t = r ln2 = th + tl
    const float th = __fmul_rn(rh, kLn2FHi);
    const float tl = fmaf(rl, kLn2FHi, fmaf(rh, kLn2FLo, fmaf(rh, kLn2FHi, -th)));
    // e^t - 1 = ph + pl
    const float p2 = __fmul_rn(th, th);
    const float e2 = fmaf(th, th, -p2);                           // th^2 = p2 + e2 exactly
    const float h = __fmul_rn(0.5f, p2);
    const float ph = __fadd_rn(th, h);
    const float l0 = __fsub_rn(h, __fsub_rn(ph, th));             // fast two-sum, |th| >= |h|
    const float c34 = __fmul_rn(p2, fmaf(th, kInv6F, __fmul_rn(p2, kInv24F)));   // t^3/6 + t^4/24
    const float pl = __fadd_rn(l0, __fadd_rn(tl, fmaf(0.5f, e2, fmaf(th, tl, c34))));
    return Exp2Red{k, ph, pl};
}

__device__ __forceinline__ Exp2Red exp2_reduce(double a)
{
    const float a0 = narrow_trunc(a);
    float a1, a2;
    tail_floats(a, a1, a2);
    const float tf = fmaf(a0, 2048.0f, 12582912.0f);            // 1.5 * 2^23 + k
    const int k = __float_as_int(tf) - 0x4B400000;               // bits of 1.5 * 2^23
    const float w = fmaf(tf, -0x1p-11f, 6144.0f);                // -k/2048, exact
    const float s = __fadd_rn(a0, w);                             // a0 - k/2048, exact
    // r = s + a1 + a2: two-sum of s and a1, then the small a2
    const float rh = __fadd_rn(s, a1);
    const float bb = __fsub_rn(rh, s);
    const float rl = __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(rh, bb)), __fsub_rn(a1, bb)), a2);
    return exp2_poly(k, rh, rl);
}

// 2^a for a <= 0 (finite or -inf; a <= -1021 returns 0, below four times the
// smallest normal double), table-driven after Tang (ACM TOMS 1989) in base 2:
// with k = round(2048 a) and r = a - k/2048, 2^a = 2^(k >> 11) *
// 2^((k & 2047)/2048) * 2^r, in two forms that return the same bits:
// exp2_tab_int uses no FP64 operation (for kernels bound by the FP64 pipe),
// exp2_tab_fp uses two (for kernels whose FP32 and integer pipes are busy).
// Both carry the reduction and 2^r - 1 in float pairs (exp2_reduce):
//  - a is split exactly into three floats, a0 = a truncated to 24 bits
//    (narrow_trunc) and the tail a1 + a2 (tail_floats);
//  - k is found from a0 (2048 |a0| < 2^22, so adding 1.5 * 2^23 rounds it to
//    an integer); -k/2048 is exact in float, and so is s = a0 - k/2048 (both
//    are multiples of a0's ulp and |s| <= 2^-12 + 2^-23 |a|);
//  - r = s + a1 + a2 as a float pair (rh, rl) by Knuth's two-sum, exact up
//    to the rounding of rl (below 2^-60 absolute);
//  - t = r ln2 as a float pair from ln2 = hi + lo (Dekker's product with an
//    FMA), and e^t - 1 = t + t^2/2 + t^3/6 + t^4/24 as a float pair (ph, pl):
//    t^2/2 with its exact product error, the t^3 and t^4 terms in float;
//    |t| <= 2.6e-4 for |a| <= 1021, so the omitted t^5/120 is below 2e-21
//    and the pair is within ~2^-59 of 2^r - 1.
// Then P = trunc(ph) + trunc(pl), each truncated toward zero to a multiple of
// 2^-63 (|P| < 2^-11, so P is a multiple of 2^-63 below 2^52 of them: exact
// in FP64 and in a 64-bit integer), and the result is T (1 + P) rounded to
// nearest even, T = 2^((k & 2047)/2048) from the 2048-entry table, scaled by
// 2^(k >> 11) on the exponent field.  Error against 2^a: table and final
// rounding 0.5 ulp each plus ~0.03 ulp, under 1.05 ulp over the whole range;
// the blob terms use -58.5 <= a <= 0.
// 2^(k/2048) (1 + ph + pl) for a reduction e with k >> 11 >= -1021: one FP64
// addition (exact) and one FMA.
__device__ __forceinline__ double exp2_scale_fp(const Exp2Red &e, const double *__restrict__ T)
{
    const double P = __dadd_rn(widen(trunc63(e.ph)), widen(trunc63(e.pl)));   // exact
    const double Tj = T[e.k & (kExpTabN - 1)];
    const double v = fma(Tj, P, Tj);                                         // RN(T (1 + P))
    return __hiloint2double(__double2hiint(v) + ((e.k >> 11) << 20), __double2loint(v));
}

__device__ __forceinline__ double exp2_tab_fp(double a, const double *__restrict__ T)
{
    const double v = exp2_scale_fp(exp2_reduce(a), T);
    const unsigned ahi = (unsigned)__double2hiint(a);
    // a <= -1021 (sign set, |a| >= 1021: hi word >= that of -1021.0), -inf and
    // NaN with the sign bit set flush to 0
    return ahi >= 0xC08FE800u ? 0.0 : v;
}

// The same value in 64-bit integer arithmetic: with T = S 2^-52 (S its 53-bit
// significand, T in [1, 2)) and U = 2^63 + P 2^63, T (1 + P) = S U 2^-115
// exactly; the 117-bit product S U (high and low 64-bit words) is normalised
// by its leading zeros and rounded to 53 bits, to nearest with ties to even
// (round bit and sticky bits), as the FMA of exp2_tab_fp rounds it.
__device__ __forceinline__ double exp2_scale_int(const Exp2Red &e, const double *__restrict__ T)
{
    const long long P = fix63(e.ph) + fix63(e.pl);                   // exact, |P| < 2^52
    const unsigned long long tb = (unsigned long long)__double_as_longlong(T[e.k & (kExpTabN - 1)]);
    const unsigned long long S = (tb & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const unsigned long long U = 0x8000000000000000ull + (unsigned long long)P;
    const unsigned long long hi = __umul64hi(S, U), lo = S * U;     // S U < 2^117
    const int lz = __clzll((long long)hi) - 11;                      // 0, 1 or 2
    const unsigned long long m = lz == 0 ? hi : (hi << lz) | (lo >> (64 - lz));
    const unsigned long long r = lo << lz;                            // round bit, then sticky bits
    const unsigned long long up = (r >> 63) & ((r << 1) != 0ull ? 1ull : (m & 1ull));
    const long long bits = ((long long)(1023 - lz + (e.k >> 11)) << 52) + (long long)(m + up);
    return __longlong_as_double(bits);
}

__device__ __forceinline__ double exp2_tab_int(double a, const double *__restrict__ T)
{
    const double v = exp2_scale_int(exp2_reduce(a), T);
    const unsigned ahi = (unsigned)__double2hiint(a);
    return ahi >= 0xC08FE800u ? 0.0 : v;
}

// u^2 for |u| < 8 in 64-bit fixed point, in units of 2^-56, within one unit,
// and the largest biased exponent seen in emax.  U = |u| 2^60 is formed from
// u's significand M by a shift, M 2^(e - 1015) (exact for |u| >= 2^-8; below
// that truncated by less than 2^-60, which moves u^2 by less than 2^-67), and
// split as U = H 2^32 + L (H < 2^31); then U^2 2^-64 = H^2 + (H L + L^2
// 2^-33) 2^-31 + (under 2^-32), the middle term rounded to nearest: two
// 32 x 32 -> 64-bit products and one high half.  Larger e only raise emax
// (the caller culls them); the sum of three such squares stays below 2^64.
__device__ __forceinline__ unsigned long long sq_fix56(double u, unsigned &emax)
{
    const unsigned hi = (unsigned)__double2hiint(u), lo = (unsigned)__double2loint(u);
    const unsigned e = (hi >> 20) & 0x7FFu;
    const unsigned long long M = ((unsigned long long)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
    const int sh = (int)e - 1015;
    const unsigned long long U = sh >= 0 ? M << min(sh, 10) : M >> min(-sh, 63);   // zero, subnormal: 0
    const unsigned H = (unsigned)(U >> 32), L = (unsigned)U;
    const unsigned long long HL = (unsigned long long)H * L + (__umulhi(L, L) >> 1) + (1ull << 30);
    emax = max(emax, e);
    return (unsigned long long)H * H + (HL >> 31);
}

// |u|^2 = 58.5 (the cull threshold kBlobCull2) in units of 2^-56.
constexpr unsigned long long kBlobCullQ56 = 0x3A80000000000000ull;

// The Gaussian of a blob term, G = 2^(-|u|^2) for FP64 u = (u0, u1, u2),
// with the exponent formed without FP64 operations: |u|^2 is summed in
// 64-bit fixed point (sq_fix56, within 2^-55.4 of the exact sum of the
// squares of the given u, where the FP64 form rounds |u|^2 to 53 bits, up
// to 2^-47 for |u|^2 near 58); k = round(2048 |u|^2) and r = k/2048 - |u|^2
// (|r| <= 2^-12) come from its bits, r as a float pair (its bits down to
// 2^-34 and the rest, both exact), and 2^r, the table entry and the scaling
// follow exp2_poly and exp2_scale_int (or exp2_scale_fp: the same bits).
// Error against the exact 2^(-|u|^2) of the given u below 1.05 ulp (CPU
// emulation of these steps against exact rationals, and the GPU test).
// Returns +0 for a negligible term (|u|^2 >= 58.5, or some |u_i| >= 8) and a
// NaN if some u_i is infinite or NaN.
__device__ __forceinline__ double blob_gauss(double u0, double u1, double u2, const double *__restrict__ T,
                                             bool exp_fp)
{
    unsigned emax = 0u;
    const unsigned long long q = sq_fix56(u0, emax) + sq_fix56(u1, emax) + sq_fix56(u2, emax);
    if (emax >= 1026u) return emax == 2047u ? __longlong_as_double(0x7FF8000000000000ll) : 0.0;
    if (q >= kBlobCullQ56) return 0.0;
    const long long K = (long long)((q + (1ull << 44)) >> 45);      // round(2048 |u|^2)
    const long long ra = (K << 45) - (long long)q;                  // r in units of 2^-56, |ra| <= 2^44
    const int vh = (int)(ra >> 22);                                 // |vh| <= 2^22
    const unsigned vl = (unsigned)ra & 0x3FFFFFu;
    // small integers as floats by the bias trick (exact), then scaled
    const float rh = __fmul_rn(__fsub_rn(__int_as_float(0x4B400000 + vh), 12582912.0f), 0x1p-34f);
    const float rl = __fmul_rn(__fsub_rn(__uint_as_float(0x4B000000u | vl), 8388608.0f), 0x1p-56f);
    const Exp2Red e = exp2_poly(-(int)K, rh, rl);
    return exp_fp ? exp2_scale_fp(e, T) : exp2_scale_int(e, T);
}

// 2^a in FP32 with the hardware base-2 exponential (ex2.approx.ftz.f32:
// relative error ~2^-22, subnormal results flushed to zero).
__device__ __forceinline__ float exp2_fast(float a)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// True if v is neither infinite nor NaN, tested on the high word (integer pipe).
__device__ __forceinline__ bool finite_bits(double v)
{
    return (~(unsigned)__double2hiint(v) & 0x7ff00000u) != 0u;
}

// v > 0 (+inf included; NaN, zeros and negatives excluded).  For a double
// the decision is an unsigned compare of the bit pattern, off the FP64 pipe.
__device__ __forceinline__ bool positive(double v)
{
    return (unsigned long long)__double_as_longlong(v) - 1ull < 0x7FF0000000000000ull;
}
__device__ __forceinline__ bool positive(float v) { return v > 0.0f; }

// fmax(m, |d|) for m >= 0 (NaN operands ignored as fmax ignores them); for a
// double on the bit patterns (non-negative doubles order as their patterns).
__device__ __forceinline__ double max_abs(double m, double d)
{
    const unsigned long long a = (unsigned long long)__double_as_longlong(d) & 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long b = (unsigned long long)__double_as_longlong(m);
    constexpr unsigned long long kInf = 0x7FF0000000000000ull;
    return (a > b || b > kInf) && a <= kInf ? __longlong_as_double((long long)a) : m;
}
__device__ __forceinline__ float max_abs(float m, float d) { return fmaxf(m, fabsf(d)); }

// 1/v of either sign in precision R: recip_pos on |v| for double (an FP64
// division is ~10 FP64-pipe operations), the correctly rounded float reciprocal
// for float.  v = 0 gives inf of v's sign; v NaN gives NaN.
template <typename R>
__device__ __forceinline__ R recip(R v);
template <>
__device__ __forceinline__ double recip<double>(double v)
{
    return copysign(recip_pos(fabs(v)), v);
}
template <>
__device__ __forceinline__ float recip<float>(float v)
{
    return __frcp_rn(v);
}

template <typename R>
__device__ __forceinline__ const R *blob_table(const MediumParams &m);
template <>
__device__ __forceinline__ const double *blob_table<double>(const MediumParams &m) { return m.blobs64s; }
template <>
__device__ __forceinline__ const float *blob_table<float>(const MediumParams &m) { return m.blobs32; }

// Stage the scaled blob rows the evaluator of precision R reads into shared
// memory (all threads of the block call it).  FP64: row after row.  FP32:
// pairs of blobs interleaved field by field, (f_2p, f_2p+1) as one float2 per
// field, for the packed FP32x2 evaluator; an odd count is padded with a zero
// row (zero amplitude: it adds exactly nothing).
template <typename R>
__device__ __forceinline__ void stage_blobs(const MediumParams &m, R *sb)
{
    const R *src = blob_table<R>(m);
    if constexpr (sizeof(R) == 8) {
        for (int j = threadIdx.x; j < m.n_blobs * kBlobStride; j += blockDim.x) sb[j] = src[j];
    } else {
        const int np = (m.n_blobs + 1) / 2;
        for (int e = threadIdx.x; e < np * 2 * kBlobStride; e += blockDim.x) {
            const int p = e / (2 * kBlobStride), f = (e / 2) % kBlobStride, h = e & 1;
            const int j = 2 * p + h;
            sb[e] = j < m.n_blobs ? src[kBlobStride * j + f] : (R)0;
        }
    }
}

// A 16-byte shared-memory load as one instruction (p 16-byte aligned, in
// shared memory).
__device__ __forceinline__ float4 lds128(const float4 *p)
{
    float4 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

// Packed FP32x2 arithmetic (two lanes of float per instruction on sm_100 and
// later, the compiler's builtins): d = a b + c and a b, each half correctly
// rounded; neg2 negates both halves.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Blob terms whose exponent is below this are skipped.  The FP64, FP32 and
// double-float evaluators' rows carry the exponent in base 2 (sigma =
// 1/sqrt(2 w^2 ln2), s2 = s/ln2), so that a term is A 2^(-|u|^2): the
// threshold 2^-58.5 = e^-40.55 leaves a contribution below 2.6e-18 |A| to
// n^2 (and below 3e-17 |A| / w to grad n^2 for the widths in use), far below
// the rounding of the sums.
constexpr double kBlobCull2 = -58.5;
// FP32 pre-test of the FP64 evaluator: a term whose |u|^2, computed in FP32
// from x (truncated, relative error 2^-23) and rounded sigma, sigma c
// (2^-24), exceeds 59 has an exact exponent below -58.5.  The error of each
// u_i is below 6e-8 (3 sigma |x_i| + sigma |c_i| + |u_i|), that of |u|^2
// (|u| < 7.7 near the threshold) below 27 times that; the host sets pre_lim
// so that sigma (2 max|x_i| + max|c_i|) <= 1e5 for every blob, which keeps
// the error below 0.2, under the 0.5 margin.  The FP64 test then decides the
// remaining terms exactly as without the pre-test; rays beyond pre_lim skip
// the pre-test.
constexpr float kBlobCullQF2 = 59.0f;

// Evaluation context: the shared exp table, the FP32 pre-test rows (FP64
// path with a block-shared table only), the double-float tables (GF_F64X) and
// a live-term counter.
template <typename R>
struct EvalCtx {
    const double *T = nullptr;   // 2^(j/2048) table (FP64 path)
    const float *pre = nullptr;  // FP32 pre-test rows, 4 floats per blob, or NULL
    int pre_stride = 1;          // field f of blob j at pre[(4 j + f) * pre_stride]
    const float *dfb = nullptr;  // double-float blob rows (GF_F64X mode)
    const float *dfT = nullptr;  // double-float 2^(j/64) table (GF_F64X mode)
    int live = 0;                // blob terms evaluated (work counter)
    bool exp_fp = false;         // blob exponentials by exp2_tab_fp (else exp2_tab_int; same bits)
};

// Stage the FP32 pre-test rows (sigma, -sigma c).
__device__ __forceinline__ void stage_pretest(const MediumParams &m, float *sp)
{
    for (int j = threadIdx.x; j < m.n_blobs * 4; j += blockDim.x) sp[j] = m.pre32[j];
}

// The point of an FP32 pre-test: truncated coordinates, and whether the
// pre-test is valid there (max_i |x_i| <= pre_lim).
struct PreX {
    float x0, x1, x2;
    bool on;
};

__device__ __forceinline__ PreX pretest_point(const MediumParams &m, const double *x)
{
    PreX p;
    p.x0 = narrow_trunc(x[0]);
    p.x1 = narrow_trunc(x[1]);
    p.x2 = narrow_trunc(x[2]);
    p.on = fmaxf(fabsf(p.x0), fmaxf(fabsf(p.x1), fabsf(p.x2))) <= m.pre_lim;
    return p;
}

// True if the blob whose pre-test row is bp (field f at bp[f * ps]) is
// certainly negligible at p (see kBlobCullQF2); p.on must hold.
__device__ __forceinline__ bool pretest_negligible(const float *__restrict__ bp, int ps, const PreX &p)
{
    const float v0 = fmaf(bp[0], p.x0, bp[ps]), v1 = fmaf(bp[0], p.x1, bp[2 * ps]), v2 = fmaf(bp[0], p.x2, bp[3 * ps]);
    return v0 * v0 + v1 * v1 + v2 * v2 > kBlobCullQF2;
}

// One Gaussian-blob term on a scaled row b (field f at b[f * stride]):
// u = sigma x - sigma c with sigma = 1/sqrt(2 w^2 ln2), G = 2^(-|u|^2) =
// exp(s |x - c|^2); for a term that is not negligible (exponent >= -58.5)
// adds A G to n2 and (-2 ln2 sigma A) G u (= 2 s A G (x - c)) to g and counts
// it in live.  Returns G, or 0 for a negligible term.
__device__ __forceinline__ double blob_term_scaled(const double *__restrict__ b, int stride, const double *x,
                                                   double &n2, double *g, const double *__restrict__ T, int &live,
                                                   bool exp_fp)
{
    const double sg = b[0];
    const double u0 = fma(sg, x[0], b[stride]), u1 = fma(sg, x[1], b[2 * stride]),
                 u2 = fma(sg, x[2], b[3 * stride]);
    const double G = blob_gauss(u0, u1, u2, T, exp_fp);
    if (__double_as_longlong(G) == 0ll) return 0.0;
    n2 = fma(b[4 * stride], G, n2);
    const double c = b[5 * stride] * G;
    g[0] = fma(c, u0, g[0]);
    g[1] = fma(c, u1, g[1]);
    g[2] = fma(c, u2, g[2]);
    ++live;
    return G;
}

// Squared index n^2 and its gradient for an isotropic medium of kind KIND plus
// the Gaussian blobs in sb:  n^2 += A exp(s q),  grad += 2 s A exp(s q) (x - c),
// with q = |x - c|^2 and s = -1 / (2 w^2).  sb holds the rows stage_blobs<R>
// stages; field f of blob j is read from sb[(kBlobStride * j + f) * stride]
// (stride 1: a table shared by the block; stride = block size: one table per
// thread).
// |x|^2 with the roundings fixed (for double: the products and sums as
// explicit fused operations), so that every kernel that evaluates the same
// point -- the forward trace and the adjoint's recomputation of it --
// obtains the same bits whatever the compiler contracts elsewhere.
template <typename R>
__device__ __forceinline__ R norm2_fixed(const R *x)
{
    if constexpr (sizeof(R) == 8)
        return fma(x[2], x[2], fma(x[1], x[1], __dmul_rn(x[0], x[0])));
    else
        return x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
}

template <typename R, int KIND>
__device__ __forceinline__ void iso_index(const MediumParams &m, const R *__restrict__ sb, int nb,
                                          const R *x, R &n2, R *g, EvalCtx<R> &cx, int stride = 1)
{
    if constexpr (KIND == K_HOMOG) {
        n2 = (R)m.n_h2;
        g[0] = g[1] = g[2] = (R)0;
    } else if constexpr (KIND == K_LUNEBURG) {
        R r2 = norm2_fixed(x);
        // r2 <= 1; for a double (r2 >= +0 or NaN) decided on the bit pattern
        bool inside;
        if constexpr (sizeof(R) == 8)
            inside = (unsigned long long)__double_as_longlong(r2) <= 0x3FF0000000000000ull;
        else
            inside = r2 <= (R)1;
        if (inside) {
            n2 = (R)2 - r2;
            g[0] = (R)-2 * x[0];
            g[1] = (R)-2 * x[1];
            g[2] = (R)-2 * x[2];
        } else {
            n2 = (R)1;
            g[0] = g[1] = g[2] = (R)0;
        }
    } else if constexpr (KIND == K_QUADRATIC) {
        R r2 = norm2_fixed(x);
        n2 = (R)2 - r2;
        g[0] = (R)-2 * x[0];
        g[1] = (R)-2 * x[1];
        g[2] = (R)-2 * x[2];
    } else {  // K_GRIN
        R c = (R)m.n02a2;
        if constexpr (sizeof(R) == 8)
            n2 = fma(-c, fma(x[2], x[2], __dmul_rn(x[1], x[1])), m.n02);
        else
            n2 = (R)m.n02 - c * (x[1] * x[1] + x[2] * x[2]);
        g[0] = (R)0;
        g[1] = (R)-2 * c * x[1];
        g[2] = (R)-2 * c * x[2];
    }
    if constexpr (sizeof(R) == 8) {
        // scaled rows: u = sigma x - sigma c, G = 2^(-|u|^2),
        // n^2 += A G, grad n^2 += (-2 ln2 sigma A) G u   (8 FP64 operations per live term:
        // u 3, n^2 1, the weight 1, grad n^2 3; G on the integer and FP32 pipes)
        PreX px = {0.f, 0.f, 0.f, false};
        if (cx.pre != nullptr) px = pretest_point(m, x);
        // one term per iteration: the trace kernels inline this loop once per
        // stage, and a longer body makes the instruction cache miss
#pragma unroll 1
        for (int j = 0; j < nb; ++j) {
            if (px.on && pretest_negligible(cx.pre + 4 * j * cx.pre_stride, cx.pre_stride, px)) continue;
            blob_term_scaled(sb + kBlobStride * j * stride, stride, x, n2, g, cx.T, cx.live, cx.exp_fp);
        }
    } else {
        // the same scaled form in FP32 with the hardware base-2 exponential
        // (relative error ~2^-22), two blobs per packed FP32x2 instruction
        // over the pair-interleaved rows of stage_blobs<float> (stride 1).
        // Every term is evaluated: a term below 2^-58.5 (the FP64 evaluator's
        // cut) is ~2^-34 of an FP32 ulp of n^2, and ex2 of a very negative
        // exponent flushes to zero, so no lane waits on another's terms.
        // Near a blob centre u = sigma x - sigma c loses ~ulp(sigma x) to
        // cancellation, a relative error of ~4e-6 in G there: below one float
        // ulp of n^2 for the amplitudes in use, far inside the FP32 gate.
        const float2 X0 = make_float2(x[0], x[0]), X1 = make_float2(x[1], x[1]), X2 = make_float2(x[2], x[2]);
        float2 N = make_float2(0.f, 0.f), H0 = N, H1 = N, H2 = N;
        // a pair's six float2 fields are 48 bytes: three 16-byte loads (sb is
        // a 16-byte aligned shared array)
        const float4 *rp = reinterpret_cast<const float4 *>(sb);
        const int np = (nb + 1) / 2;
#pragma unroll 2
        for (int p = 0; p < np; ++p) {
            const float4 r0 = lds128(rp + 3 * p), r1 = lds128(rp + 3 * p + 1), r2 = lds128(rp + 3 * p + 2);
            const float2 sg = make_float2(r0.x, r0.y);
            const float2 u0 = fma2(sg, X0, make_float2(r0.z, r0.w)), u1 = fma2(sg, X1, make_float2(r1.x, r1.y)),
                         u2 = fma2(sg, X2, make_float2(r1.z, r1.w));
            const float2 nq = fma2(neg2(u2), u2, fma2(neg2(u1), u1, mul2(neg2(u0), u0)));   // -|u|^2
            const float2 G = make_float2(exp2_fast(nq.x), exp2_fast(nq.y));
            N = fma2(make_float2(r2.x, r2.y), G, N);
            const float2 c = mul2(make_float2(r2.z, r2.w), G);
            H0 = fma2(c, u0, H0);
            H1 = fma2(c, u1, H1);
            H2 = fma2(c, u2, H2);
        }
        n2 += N.x + N.y;
        g[0] += H0.x + H0.y;
        g[1] += H1.x + H1.y;
        g[2] += H2.x + H2.y;
        cx.live += nb;
    }
}

// Ray right-hand side for an isotropic medium, D = |k|^2 - w^2 n^2:
//   f_x = -D_k / D_w = k / (w n^2),  f_k = D_x / D_w = w grad n^2 / (2 n^2).
// Returns false (cut-off) where n^2 <= 0.  D is computed when WANT_D.
template <typename R>
struct Omega {
    R w, inv_w, half_w, inv_w2;   // w, 1/w, w/2, 1/w^2
};

// ng, if not NULL, receives n^2 and grad n^2 (the adjoint's stage values).
// The right-hand side from n^2 and grad n^2 at y (D when WANT_D), with the
// roundings fixed for double, shared by every isotropic evaluator.
template <typename R, bool WANT_D>
__device__ __forceinline__ bool rhs_iso_from_index(const Omega<R> &om, const R *y, R n2, const R *g, R *f, R &D)
{
    if constexpr (WANT_D) {
        if constexpr (sizeof(R) == 8)
            D = fma(-__dmul_rn(om.w, om.w), n2, norm2_fixed(y + 3));
        else
            D = y[3] * y[3] + y[4] * y[4] + y[5] * y[5] - om.w * om.w * n2;
    }
    if (!positive(n2)) return false;
    R inv;
    if constexpr (sizeof(R) == 8)
        inv = recip_pos(n2);
    else   // the hardware reciprocal (within one ulp; n^2 is far from the subnormals)
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(n2));
    const R a = inv * om.inv_w;
    const R b = om.half_w * inv;
    f[0] = a * y[3];
    f[1] = a * y[4];
    f[2] = a * y[5];
    f[3] = b * g[0];
    f[4] = b * g[1];
    f[5] = b * g[2];
    return true;
}

template <typename R, int KIND, bool WANT_D>
__device__ __forceinline__ bool rhs_iso(const MediumParams &m, const R *__restrict__ sb, int nb,
                                        const Omega<R> &om, const R *y, R *f, R &D, EvalCtx<R> &cx,
                                        int stride = 1, R *ng = nullptr)
{
    R n2, g[3];
    iso_index<R, KIND>(m, sb, nb, y, n2, g, cx, stride);
    if (ng != nullptr) {
        ng[0] = n2;
        ng[1] = g[0];
        ng[2] = g[1];
        ng[3] = g[2];
    }
    return rhs_iso_from_index<R, WANT_D>(om, y, n2, g, f, D);
}

// Periodic tricubic B-spline: values and gradients of the 7 channels
// (M11 M12 M13 M22 M23 M33 eps) at x, arithmetic in R.  Uniform cubic
// B-spline weights of nodes i-1..i+2 at fraction f:
//   (1-f)^3/6, (3f^3 - 6f^2 + 4)/6, (-3f^3 + 3f^2 + 3f + 1)/6, f^3/6,
// evaluated separably: x first, then y and z.
template <typename R>
__device__ __forceinline__ void bspline_w(R f, R inv_h, R *B, R *dB)
{
    R u = (R)1 - f;
    R f2 = f * f, f3 = f2 * f;
    const R s6 = (R)1 / (R)6;
    B[0] = u * u * u * s6;
    B[1] = ((R)3 * f3 - (R)6 * f2 + (R)4) * s6;
    B[2] = ((R)-3 * f3 + (R)3 * f2 + (R)3 * f + (R)1) * s6;
    B[3] = f3 * s6;
    dB[0] = (R)-0.5 * u * u * inv_h;
    dB[1] = ((R)1.5 * f2 - (R)2 * f) * inv_h;
    dB[2] = ((R)-1.5 * f2 + f + (R)0.5) * inv_h;
    dB[3] = (R)0.5 * f2 * inv_h;
}

// Grid value as R.  For double the widening float -> double is done on the
// bit pattern with integer operations (exact: the exponent is re-biased by
// 1023 - 127 and the significand gains 29 zero bits), which keeps the 28
// conversions of every grid row off the FP64 pipe.  Valid for zeros and
// normal floats: the device copy of the grid holds no subnormal, infinite or
// NaN value (gf_medium_create rejects non-finite values and flushes
// subnormals to zero).
template <typename R>
__device__ __forceinline__ R grid_value(float v);
template <>
__device__ __forceinline__ float grid_value<float>(float v) { return v; }
template <>
__device__ __forceinline__ double grid_value<double>(float v)
{
    const unsigned b = __float_as_uint(v);
    const unsigned mag = b & 0x7FFFFFFFu;
    const unsigned hi = (b & 0x80000000u) | ((mag >> 3) + (mag != 0u ? (1023u - 127u) << 20 : 0u));
    return __hiloint2double((int)hi, (int)(b << 29));
}

template <typename R>
__device__ __forceinline__ void spline_fields(const MediumParams &m, const R *x, R *val, R (*grad)[3])
{
    const int n = m.grid_n;
    const R inv_h = (R)n * (R)0.5;
    int base[3];
    R B[3][4], dB[3][4];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        R u = (x[ax] + (R)1) * inv_h;
        R fl = floor(u);
        // wrap the integer cell index into [0, n) once; neighbours wrap below
        long long ib = (long long)fl;
        long long r = ib % n;
        base[ax] = (int)(r < 0 ? r + n : r);
        bspline_w<R>(u - fl, inv_h, B[ax], dB[ax]);
    }
#pragma unroll
    for (int ch = 0; ch < 7; ++ch) val[ch] = grad[ch][0] = grad[ch][1] = grad[ch][2] = (R)0;
    int ix[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int v = base[0] - 1 + a;
        ix[a] = v < 0 ? v + n : (v >= n ? v - n : v);
    }
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
        int iz = base[2] - 1 + c;
        iz = iz < 0 ? iz + n : (iz >= n ? iz - n : iz);
#pragma unroll 1
        for (int b = 0; b < 4; ++b) {
            int iy = base[1] - 1 + b;
            iy = iy < 0 ? iy + n : (iy >= n ? iy - n : iy);
            const float4 *row = m.grid + 2 * ((int64_t)(iz * n + iy) * n);
            R sx[7], dsx[7];
#pragma unroll
            for (int ch = 0; ch < 7; ++ch) sx[ch] = dsx[ch] = (R)0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                float4 lo = __ldg(row + 2 * ix[a]);
                float4 hi = __ldg(row + 2 * ix[a] + 1);
                R v[7] = {grid_value<R>(lo.x), grid_value<R>(lo.y), grid_value<R>(lo.z), grid_value<R>(lo.w),
                          grid_value<R>(hi.x), grid_value<R>(hi.y), grid_value<R>(hi.z)};
#pragma unroll
                for (int ch = 0; ch < 7; ++ch) {
                    sx[ch] += B[0][a] * v[ch];
                    dsx[ch] += dB[0][a] * v[ch];
                }
            }
            R w = B[1][b] * B[2][c], wy = dB[1][b] * B[2][c], wz = B[1][b] * dB[2][c];
#pragma unroll
            for (int ch = 0; ch < 7; ++ch) {
                val[ch] += w * sx[ch];
                grad[ch][0] += w * dsx[ch];
                grad[ch][1] += wy * sx[ch];
                grad[ch][2] += wz * sx[ch];
            }
        }
    }
}

// Ray right-hand side for D = k^T M k - w^2 eps:
//   f_x = -D_k / D_w = M k / (w eps),
//   f_k =  D_x / D_w = -(k^T dM k - w^2 d eps) / (2 w eps).
template <typename R>
__device__ __forceinline__ bool rhs_spline(const MediumParams &m, const Omega<R> &om, const R *y, R *f, R &D)
{
    const R omega = om.w;
    R val[7], grad[7][3];
    spline_fields<R>(m, y, val, grad);
    const R *k = y + 3;
    R Mk0 = val[0] * k[0] + val[1] * k[1] + val[2] * k[2];
    R Mk1 = val[1] * k[0] + val[3] * k[1] + val[4] * k[2];
    R Mk2 = val[2] * k[0] + val[4] * k[1] + val[5] * k[2];
    R eps = val[6];
    D = k[0] * Mk0 + k[1] * Mk1 + k[2] * Mk2 - omega * omega * eps;
    if (!(eps > (R)0)) return false;
    R inv = (R)1 / (omega * eps);
    f[0] = Mk0 * inv;
    f[1] = Mk1 * inv;
    f[2] = Mk2 * inv;
    R h = (R)-0.5 * inv;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        R kMk = grad[0][c] * k[0] * k[0] + grad[3][c] * k[1] * k[1] + grad[5][c] * k[2] * k[2] +
                (R)2 * (grad[1][c] * k[0] * k[1] + grad[2][c] * k[0] * k[2] + grad[4][c] * k[1] * k[2]);
        f[3 + c] = (kMk - omega * omega * grad[6][c]) * h;
    }
    return true;
}

// Cold magnetised plasma (B along z, slab profiles along x), Stix form of
// det(eps + n n - n^2 I) with n = k / w and its gradients by the chain rule:
// D_k through a = (k_x^2 + k_y^2)/w^2 and b = k_z^2/w^2, D_x through
// S, Dst, P (f, g depend on x_0), D_w through a, b, S, Dst, P.  The ray
// equations need only D_k, D_x and D_w; D_w = 0 is the cut-off test.
// Per species t = wp2 / (w^2 - W^2) (wp2 = w_p^2 f, W = Omega g) enters
// S = 1 - sum t and Dst = sum W t / w; its derivatives are
// t_x = (wp2_x + 2 W t W_x) / den and t_w = -2 w t / den, so
//   S_x = -sum t_x,  Dst_x = sum (W_x t + W t_x) / w,
//   S_w = 2 w sum t / den,  Dst_w = -(sum W t / w^2 + 2 sum W t / den),
// and P = 1 - f sum(w_p^2) / w^2 is linear in f: P_x, P_w follow from the one
// sum.  The factors 1/w, 2w common to the species are applied once, after the
// loop; wp2_x = w_p^2 f', W_x = Omega g' and 2 W_x are the host's constants.
template <typename R, bool WANT_D = true>
__device__ __forceinline__ bool rhs_cold(const MediumParams &m, const Omega<R> &om, const R *y, R *f, R &D)
{
    const R w = om.w, w2 = w * w, iw2 = om.inv_w2;
    const R fx = (R)m.prof[1];
    const R fv = fma(fx, y[0], (R)m.prof[0]), gv = fma((R)m.prof[3], y[0], (R)m.prof[2]);
    R S = 1, Sx = 0, sWt = 0, sDx = 0, sT2 = 0, sWT2 = 0;
    for (int sp = 0; sp < m.n_species; ++sp) {
        const R wp2 = (R)m.species[2 * sp] * fv, W = (R)m.species[2 * sp + 1] * gv;
        const R wp2x = (R)m.cold_x[3 * sp], Wx = (R)m.cold_x[3 * sp + 1], Wx2 = (R)m.cold_x[3 * sp + 2];
        const R den = fma(-W, W, w2);
        const R iden = recip<R>(den);   // either sign: below or above the cyclotron resonance
        const R t = wp2 * iden, Wt = W * t;
        const R tx = fma(wp2x, iden, (Wt * Wx2) * iden);
        S -= t;
        Sx -= tx;
        sWt += Wt;
        sDx = fma(Wx, t, fma(W, tx, sDx));
        sT2 = fma(t, iden, sT2);
        sWT2 = fma(Wt, iden, sWT2);
    }
    const R Dst = sWt * om.inv_w, Dx = sDx * om.inv_w;
    const R Sw = (R)2 * w * sT2;
    const R Dw = -fma(sWt, iw2, (R)2 * sWT2);
    const R Pc = (R)m.wp_sum * iw2;
    const R P = fma(-Pc, fv, (R)1), Px = -Pc * fx, Pw = ((R)2 * om.inv_w * Pc) * fv;
    const R a = fma(y[4], y[4], y[3] * y[3]) * iw2, b = (y[5] * y[5]) * iw2;
    const R ab = a + b, a2b = ab + b, PmA = P - a;
    const R RL = fma(S, S, -(Dst * Dst));
    // D = S a (a+b) + P b (a+b) - RL a - P S (a+2b) + P RL
    if constexpr (WANT_D) D = fma(fma(S, a, P * b), ab, fma(RL, PmA, -(P * S) * a2b));
    const R DS = fma(a, ab, fma(-P, a2b, (R)2 * S * PmA));
    const R DD = (R)-2 * Dst * PmA;
    const R DP = fma(b, ab, fma(-S, a2b, RL));
    const R Da = fma(S, a + ab, fma(P, b - S, -RL));
    const R Db = fma(P, fma((R)-2, S, a2b), S * a);
    const R Dom = fma(DP, Pw, fma(DD, Dw, fma(DS, Sw, fma(Db, b, Da * a) * ((R)-2 * om.inv_w))));
    if (!(Dom != (R)0) || !isfinite(Dom)) return false;
    const R inv = recip<R>(Dom);
    const R cA = (Da * inv) * ((R)-2 * iw2), cB = (Db * inv) * ((R)-2 * iw2);
    f[0] = cA * y[3];
    f[1] = cA * y[4];
    f[2] = cB * y[5];
    f[3] = fma(DP, Px, fma(DD, Dx, DS * Sx)) * inv;
    f[4] = (R)0;
    f[5] = (R)0;
    return true;
}

// dD/dk_x of the cold plasma (for Newton's method on k_x).
template <typename R>
__device__ __forceinline__ R cold_dkx(const MediumParams &m, const Omega<R> &om, const R *y)
{
    const R w = om.w, w2 = w * w;
    const R fv = (R)m.prof[0] + (R)m.prof[1] * y[0], gv = (R)m.prof[2] + (R)m.prof[3] * y[0];
    R S = 1, Dst = 0, P = 1;
    for (int sp = 0; sp < m.n_species; ++sp) {
        const R wp2 = (R)m.species[2 * sp] * fv, W = (R)m.species[2 * sp + 1] * gv;
        const R t = wp2 / (w2 - W * W);
        S -= t;
        Dst += W * t * om.inv_w;
        P -= wp2 / w2;
    }
    const R a = (y[3] * y[3] + y[4] * y[4]) / w2, b = y[5] * y[5] / w2;
    const R RL = S * S - Dst * Dst;
    const R Da = S * ((R)2 * a + b) + P * b - RL - P * S;
    return (R)2 * Da * y[3] / w2;
}

// The RK4 combination of the fixed-step trace, shared by the forward kernel
// and the adjoint's recomputation so that both produce the same bits: for
// double every rounding is explicit (y + a K as one fused operation,
// acc + 2 K fused, then y + h6 (acc + K4) as a rounded product and sum);
// for float the expressions the compiler contracts as it sees fit.
template <typename R>
__device__ __forceinline__ R rk_axpy(R a, R k, R y)
{
    if constexpr (sizeof(R) == 8)
        return fma(a, k, y);
    else
        return y + a * k;
}

template <typename R>
__device__ __forceinline__ R rk_acc2(R acc, R k)
{
    if constexpr (sizeof(R) == 8)
        return fma(2.0, k, acc);
    else
        return acc + (R)2 * k;
}

template <typename R>
__device__ __forceinline__ R rk_inc(R h6, R acc, R k)
{
    if constexpr (sizeof(R) == 8)
        return __dmul_rn(h6, __dadd_rn(acc, k));
    else
        return h6 * (acc + k);
}

// Dispatch on the medium kind at compile time.
template <typename R, int KIND>
struct Rhs {
    const MediumParams &m;
    const R *sb;
    int nb;
    Omega<R> om;
    template <bool WANT_D = true>
    __device__ __forceinline__ bool eval(const R *y, R *f, R &D, EvalCtx<R> &cx) const
    {
        if constexpr (KIND == K_SPLINE)
            return rhs_spline<R>(m, om, y, f, D);
        else if constexpr (KIND == K_COLD)
            return rhs_cold<R, WANT_D>(m, om, y, f, D);
        else
            return rhs_iso<R, KIND, WANT_D>(m, sb, nb, om, y, f, D, cx);
    }
};

template <typename R>
__host__ __device__ inline Omega<R> make_omega(double w)
{
    return Omega<R>{(R)w, (R)(1.0 / w), (R)(0.5 * w), (R)(1.0 / (w * w))};
}

}  // namespace gf
