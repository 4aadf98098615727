// gf_dopri5.cu -- batched adaptive Dormand-Prince 5(4) ray tracing over many
// media: a persistent work-stealing kernel with warp-level refill of finished
// lanes, a one-launch-per-medium baseline that runs the same per-ray code, the
// CUDA-graph capture of both schedules, and the launch-shape autotuner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "gf_dfloat.cuh"
#include "gf_internal.cuh"

namespace gf {

// Dormand & Prince (1980) RK5(4)7M coefficients; e = b - b* (5th minus 4th order).
namespace dp {
constexpr double a21 = 1.0 / 5.0;
constexpr double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
constexpr double a41 = 44.0 / 45.0, a42 = -56.0 / 15.0, a43 = 32.0 / 9.0;
constexpr double a51 = 19372.0 / 6561.0, a52 = -25360.0 / 2187.0, a53 = 64448.0 / 6561.0,
                 a54 = -212.0 / 729.0;
constexpr double a61 = 9017.0 / 3168.0, a62 = -355.0 / 33.0, a63 = 46732.0 / 5247.0,
                 a64 = 49.0 / 176.0, a65 = -5103.0 / 18656.0;
constexpr double a71 = 35.0 / 384.0, a73 = 500.0 / 1113.0, a74 = 125.0 / 192.0,
                 a75 = -2187.0 / 6784.0, a76 = 11.0 / 84.0;
constexpr double e1 = 35.0 / 384.0 - 5179.0 / 57600.0, e3 = 500.0 / 1113.0 - 7571.0 / 16695.0,
                 e4 = 125.0 / 192.0 - 393.0 / 640.0, e5 = -2187.0 / 6784.0 - (-92097.0 / 339200.0),
                 e6 = 11.0 / 84.0 - 187.0 / 2100.0, e7 = 0.0 - 1.0 / 40.0;
}  // namespace dp

struct Ctl {
    double rtol, atol, h0, t_max, r2, fac_min, fac_max, safety;
    int64_t max_steps, max_attempts;
    Omega<double> om;
};

// Device view of a batch.
struct BatchView {
    int32_t n_media, nb_max, n_items, pad;
    const double *blobs;        // n_media x nb_max scaled rows (kBlobStride values each)
    const float *pre;           // n_media x nb_max FP32 pre-test rows (4 floats each)
    const float *df;            // n_media x nb_max double-float rows (GF_F64X launches)
    const float *pre_lim;       // n_media: validity bound of the pre-test (MediumParams::pre_lim)
    const int32_t *nb;          // n_media
    const double *base;         // n_media x 3: n_h2, n02, n02a2
    const int32_t *item_medium; // n_items
    const int64_t *item_begin;  // n_items
    const int64_t *item_end;    // n_items
};

struct Lane {
    double y[6], K1[6];
    double t, h, fmax, dm;
    int64_t ray;
    int32_t steps, rejects, status, attempts, nb;
    // the lane's medium: scaled FP64 rows, FP32 pre-test rows (or NULL) and
    // double-float rows of the batch's tables (global memory, L1/L2-resident)
    const double *rows;
    const float *prer, *dfr;
    MediumParams mp;
};

// Block-shared exponential tables: 2^(j/2048) in FP64 or as double-float pairs.
struct Tabs {
    const double *T;
    const float *dT;
};

template <int KIND, bool DF>
struct LaneRhs {
    const Lane &L;
    const Omega<double> &om;
    const Tabs &tb;
    template <bool WANT_D = true>
    __device__ __forceinline__ bool eval(const double *y, double *f, double &D) const
    {
        if constexpr (DF) {
            int live = 0;
            return rhs_df<KIND, WANT_D>(L.mp, L.dfr, L.nb, 1, om, y, f, D, tb.dT, live);
        } else {
            EvalCtx<double> cx;
            cx.T = tb.T;
            cx.pre = L.prer;
            return rhs_iso<double, KIND, WANT_D>(L.mp, L.rows, L.nb, om, y, f, D, cx, 1);
        }
    }
};

// Load ray `ray` of medium `med` into lane L (its medium's rows are read in
// place from the batch's tables).  Returns false if the ray is not active.
template <int KIND, bool DF>
__device__ __forceinline__ bool lane_load(Lane &L, const BatchView &B, const RaysView<double> &r,
                                          int med, int64_t ray, const Tabs &tb, const Ctl &c)
{
    L.status = r.status[ray];
    if (L.status != GF_RAY_ACTIVE) return false;
    L.ray = ray;
    L.nb = B.nb[med];
    L.mp.kind = KIND;
    L.mp.n_h2 = B.base[3 * med];
    L.mp.n02 = B.base[3 * med + 1];
    L.mp.n02a2 = B.base[3 * med + 2];
    L.rows = B.blobs + (int64_t)med * B.nb_max * kBlobStride;
    L.prer = nullptr;
    L.dfr = DF ? B.df + (int64_t)med * B.nb_max * kDfBlobStride : nullptr;
    if (!DF && B.pre != nullptr) {
        L.mp.pre_lim = B.pre_lim[med];
        L.prer = B.pre + (int64_t)med * B.nb_max * 4;
    }
#pragma unroll
    for (int c2 = 0; c2 < 6; ++c2) L.y[c2] = r.y[c2 * r.ld + ray];
    L.t = r.t[ray];
    L.steps = r.steps[ray];
    L.rejects = 0;
    L.attempts = 0;
    L.dm = r.d_max ? r.d_max[ray] : 0.0;
    L.h = c.h0;
    L.fmax = c.fac_max;
    double D;
    const LaneRhs<KIND, DF> f{L, c.om, tb};
    bool ok = f.eval(L.y, L.K1, D);
    L.dm = fmax(L.dm, fabs(D));
    if (!ok) L.status = GF_RAY_CUTOFF;
    return true;
}

// Final residual and store of a lane whose ray stopped.
template <int KIND, bool DF>
__device__ __forceinline__ void lane_store(const Lane &L, const RaysView<double> &r, int32_t *rejects,
                                           const Tabs &tb, const Ctl &c)
{
    double K[6], D;
    const LaneRhs<KIND, DF> f{L, c.om, tb};
    f.eval(L.y, K, D);
    const double dm = fmax(L.dm, fabs(D));
    const int64_t i = L.ray;
#pragma unroll
    for (int c = 0; c < 6; ++c) r.y[c * r.ld + i] = L.y[c];
    r.t[i] = L.t;
    r.status[i] = L.status;
    r.steps[i] = L.steps;
    if (rejects) rejects[i] = L.rejects;
    if (r.d_res) r.d_res[i] = fabs(D);
    if (r.d_max) r.d_max[i] = dm;
}

// |v| by clearing the sign bit (an integer operation).
__device__ __forceinline__ double abs_bits(double v)
{
    return __longlong_as_double(__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFll);
}

// min and max of two positive doubles (neither NaN) on their bit patterns.
__device__ __forceinline__ double min_pos(double a, double b)
{
    return __double_as_longlong(a) < __double_as_longlong(b) ? a : b;
}
__device__ __forceinline__ double max_pos(double a, double b)
{
    return __double_as_longlong(a) > __double_as_longlong(b) ? a : b;
}

// 2^-120 <= v <= 2^120 for v >= 0, decided on the bit pattern: the range in
// which v and v^(-1/10) are normal floats.
__device__ __forceinline__ bool err2_in_range(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return b >= 0x3870000000000000ull && b <= 0x4770000000000000ull;
}

// ------------------------------------------------- warp-cooperative blob sums

// The persistent kernel's lanes hold rays at different places and times, so
// their sets of non-negligible blob terms differ: evaluated lane by lane, a
// warp spends one instruction slot per term that any of its lanes needs (the
// union), while each lane needs only its own (in the batched workload 4.6 of
// 8 terms per lane against 7.2 for the union).  Here the warp evaluates its
// lanes' terms as a packed list instead: every lane selects its terms with
// the FP32 pre-test, the (lane, blob) pairs are numbered across the warp,
// and in rounds of 32 each lane computes one pair's u = sigma x - sigma c,
// exponent and Gaussian G (the FP64 evaluator's operations, on the owner's
// point and rows); the owners then add their own terms, in blob order, with
// the same fused operations as the lane-by-lane evaluator.  The sums are
// therefore the same bits as that evaluator's, whichever lanes share a warp.
// Shared memory per warp: 32 nb_max pair slots of (G, u) and their (owner,
// blob) indices.
struct CoopWarp {
    double *res;            // [32 nb_max][4]: G, u0, u1, u2
    unsigned short *pair;   // [32 nb_max]: owner lane << 8 | blob
};

__host__ __device__ constexpr size_t coop_warp_bytes(int nb_max)
{
    return (size_t)32 * nb_max * (4 * sizeof(double) + sizeof(unsigned short));
}

__device__ __forceinline__ CoopWarp coop_warp(double *sm_dyn, int nb_max)
{
    char *base = reinterpret_cast<char *>(sm_dyn) + (threadIdx.x >> 5) * coop_warp_bytes(nb_max);
    return CoopWarp{reinterpret_cast<double *>(base),
                    reinterpret_cast<unsigned short *>(base + (size_t)32 * nb_max * 4 * sizeof(double))};
}

// Adds the blob terms of the lane's medium at x to n2 and g, cooperatively.
// All 32 lanes of the warp must call it together (warp-uniform control flow);
// lanes with part = false contribute no terms and their n2, g are left as they are.
__device__ __forceinline__ void coop_blob_sums(const Lane &L, bool part, const double *x, double &n2, double *g,
                                               const double *__restrict__ T, const CoopWarp &cw)
{
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = (int)(threadIdx.x & 31u);
    unsigned m = 0u;   // candidate terms of this lane (bit j: blob j)
    if (part) {
        PreX px = {0.f, 0.f, 0.f, false};
        if (L.prer != nullptr) px = pretest_point(L.mp, x);
        for (int j = 0; j < L.nb; ++j)
            if (!(px.on && pretest_negligible(L.prer + 4 * j, 1, px))) m |= 1u << j;
    }
    const int cnt = __popc(m);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kAll, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(kAll, incl, 31);
    if (total == 0) return;
    const int first = incl - cnt;
    for (unsigned mm = m, k = first; mm != 0u; mm &= mm - 1u, ++k)
        cw.pair[k] = (unsigned short)((lane << 8) | (__ffs(mm) - 1));
    __syncwarp(kAll);
    // rounds of 32 pairs: G and u of pair p on lane p mod 32
    const unsigned long long rows = (unsigned long long)L.rows;
    for (int base = 0; base < total; base += 32) {
        const int p = base + lane;
        const int pr = p < total ? cw.pair[p] : 0;
        const int own = pr >> 8;
        const double x0 = __shfl_sync(kAll, x[0], own), x1 = __shfl_sync(kAll, x[1], own),
                     x2 = __shfl_sync(kAll, x[2], own);
        const double *b = reinterpret_cast<const double *>(__shfl_sync(kAll, rows, own)) + kBlobStride * (pr & 255);
        if (p < total) {
            const double sg = b[0];
            const double u0 = fma(sg, x0, b[1]), u1 = fma(sg, x1, b[2]), u2 = fma(sg, x2, b[3]);
            double *r = cw.res + 4 * p;
            r[0] = blob_gauss(u0, u1, u2, T, false);
            r[1] = u0;
            r[2] = u1;
            r[3] = u2;
        }
    }
    __syncwarp(kAll);
    // the owner's terms, in blob order (a culled term has G = +0 and adds nothing)
    const double *__restrict__ rb = L.rows;
    for (unsigned mm = m, k = first; mm != 0u; mm &= mm - 1u, ++k) {
        const double *r = cw.res + 4 * k;
        const double G = r[0];
        if (__double_as_longlong(G) == 0ll) continue;
        const double *b = rb + kBlobStride * (__ffs(mm) - 1);
        n2 = fma(b[4], G, n2);
        const double c = b[5] * G;
        g[0] = fma(c, r[1], g[0]);
        g[1] = fma(c, r[2], g[1]);
        g[2] = fma(c, r[3], g[2]);
    }
    __syncwarp(kAll);   // the buffers are reused by the next evaluation
}

// The right-hand side with warp-cooperative blob sums (FP64 blob rows only);
// D is formed when want_d.
template <int KIND>
__device__ __forceinline__ bool rhs_coop(const Lane &L, bool part, const Omega<double> &om, const double *y,
                                         double *f, double &D, bool want_d, const double *T, const CoopWarp &cw)
{
    double n2, g[3];
    EvalCtx<double> base;
    iso_index<double, KIND>(L.mp, nullptr, 0, y, n2, g, base);   // the index law without blobs
    coop_blob_sums(L, part, y, n2, g, T, cw);
    return want_d ? rhs_iso_from_index<double, true>(om, y, n2, g, f, D)
                  : rhs_iso_from_index<double, false>(om, y, n2, g, f, D);
}

// Stage coefficients as a queue: after stage j (2..7) is evaluated, its K_j
// enters the accumulators of stages j+1 .. j+5 with a_{j+k, j} (zero beyond
// stage 7), and the error accumulator with e_j.  The accumulator of stage j
// is a_{j1} K_1 + ... + a_{j,j-1} K_{j-1}, summed in that order with fused
// operations, exactly as an unrolled combination would.
__constant__ double c_dp_queue[6][5] = {
    {dp::a32, dp::a42, dp::a52, dp::a62, 0.0},            // K2 into stages 3..7
    {dp::a43, dp::a53, dp::a63, dp::a73, 0.0},            // K3 into stages 4..7
    {dp::a54, dp::a64, dp::a74, 0.0, 0.0},                // K4
    {dp::a65, dp::a75, 0.0, 0.0, 0.0},                    // K5
    {dp::a76, 0.0, 0.0, 0.0, 0.0},                        // K6
    {0.0, 0.0, 0.0, 0.0, 0.0}};                           // K7 (the new state's slope)
__constant__ double c_dp_err[6] = {0.0, dp::e3, dp::e4, dp::e5, dp::e6, dp::e7};   // e_2 .. e_7

// One attempted DOPRI5 step (the step-size controller of Hairer-Norsett-Wanner
// I, Sec. II.4).  Leaves L.status != ACTIVE when the ray stops.  COOP: every
// lane of the warp calls it together and the evaluations are warp-cooperative;
// part = false marks a lane without an active ray, and a lane whose ray stops
// inside the attempt goes on evaluating without terms.  Otherwise it is called
// by active lanes alone and returns as soon as the ray stops.  The six stages
// run as one loop (a single copy of the evaluator in the code) over a queue
// of stage accumulators; the combinations are explicit fused operations, so
// both forms (and both schedules) produce the same bits.
template <int KIND, bool DF, bool COOP>
__device__ __forceinline__ void lane_attempt(Lane &L, bool part, const Tabs &tb, const Ctl &c, const CoopWarp &cw)
{
    using namespace dp;
    bool go = part;
    double hs = 0.0;
    bool last = false;
    if (go) {
        if (L.steps >= c.max_steps || L.attempts >= c.max_attempts) {
            L.status = GF_RAY_MAX_STEPS;
            go = false;
        } else if (L.t >= c.t_max) {
            L.status = GF_RAY_DONE;
            go = false;
        } else {
            ++L.attempts;
            hs = L.h;
            if (L.t + hs >= c.t_max) { hs = c.t_max - L.t; last = true; }
            if (hs < 1e-14 * fmax(1.0, fabs(L.t))) { L.status = GF_RAY_STEP_UNDERFLOW; go = false; }
        }
    }
    if constexpr (!COOP) {
        if (!go) return;
    }
    const LaneRhs<KIND, DF> f{L, c.om, tb};
    const double *y = L.y, *K1 = L.K1;
    // Q[k]: accumulator of stage j + k (k = 0: the stage evaluated next); E: error sum
    double Q[5][6], E[6], K[6], Y[6], D = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        Q[0][i] = a21 * K1[i];
        Q[1][i] = a31 * K1[i];
        Q[2][i] = a41 * K1[i];
        Q[3][i] = a51 * K1[i];
        Q[4][i] = a61 * K1[i];
        E[i] = e1 * K1[i];
    }
#pragma unroll 1
    for (int j = 0; j < 6; ++j) {   // stage j + 2
#pragma unroll
        for (int i = 0; i < 6; ++i) Y[i] = fma(hs, Q[0][i], y[i]);
        const bool want_d = j == 5;
        bool ok;
        if constexpr (COOP)
            ok = rhs_coop<KIND>(L, go, c.om, Y, K, D, want_d, tb.T, cw);
        else
            ok = want_d ? f.template eval<true>(Y, K, D) : f.template eval<false>(Y, K, D);
        if (go && !ok) {
            L.status = GF_RAY_CUTOFF;
            go = false;
        }
        if constexpr (!COOP) {
            if (!go) return;
        }
        if (j == 5) break;   // K = K7 at Y = Y7, the 5th-order solution
        // K_{j+2} into the accumulators of stages j+3 .. 7, advancing the queue
        // (Q[k] becomes stage j+3+k's); the zero coefficients (e_2, a_72 and the
        // stages beyond 7) are skipped, which changes no bit of the sums
        if (j > 0) {
#pragma unroll
            for (int i = 0; i < 6; ++i) E[i] = fma(c_dp_err[j], K[i], E[i]);
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) Q[0][i] = fma(c_dp_queue[j][0], K[i], Q[1][i]);
        if (j <= 3) {
#pragma unroll
            for (int i = 0; i < 6; ++i) Q[1][i] = fma(c_dp_queue[j][1], K[i], Q[2][i]);
        }
        if (j <= 2) {
#pragma unroll
            for (int i = 0; i < 6; ++i) Q[2][i] = fma(c_dp_queue[j][2], K[i], Q[3][i]);
        }
        if (j <= 1) {
#pragma unroll
            for (int i = 0; i < 6; ++i) Q[3][i] = fma(c_dp_queue[j][3], K[i], Q[4][i]);
        }
        if (j == 0) {
#pragma unroll
            for (int i = 0; i < 6; ++i) Q[4][i] = a71 * K1[i];   // stage 7 enters: a_71 K_1 (a_72 = 0)
        }
    }
    if (!go) return;
    double K7[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        K7[i] = K[i];
        E[i] = fma(c_dp_err[5], K[i], E[i]);
    }
    bool fin = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) fin = fin && finite_bits(Y[i]) && finite_bits(K7[i]);
    if (!fin) { L.status = GF_RAY_NONFINITE; return; }
    // The controller of the oracle (Hairer-Norsett-Wanner I, Sec. II.4) in FP64
    // accuracy: err^2 = mean_i (e_i / sc_i)^2 with sc_i = atol + rtol max(|y_i|,
    // |Y_i|), accept iff err <= 1, fac = safety err^(-1/5).  The step factor
    // must be accurate to far better than FP32: near the Luneburg surface the
    // error committed by the step that crosses it depends on where the step
    // boundaries fall, and a 1e-7 relative difference in the step sizes moves
    // the solution by more than 1e-9 there.  No FP64 division, square root or
    // power: 1/sc_i is the Newton-refined reciprocal (relative error below
    // 2^-44), the factor h^2 / 6 is applied to the sum, and err2^(-1/10) is the
    // FP32 power refined by one Newton step y <- y (1 + (1 - err2 y^10) / 10)
    // (quadratic: relative error below 6e-14 from the FP32 seed's ~1e-7);
    // outside [2^-120, 2^120], where the seed is not a normal float, the FP64 power.
    double err2 = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double sc = fma(c.rtol, max_abs(abs_bits(y[i]), Y[i]), c.atol);
        const double q = E[i] * recip_pos_q(sc);
        err2 = fma(q, q, err2);
    }
    err2 = err2 * ((hs * hs) * (1.0 / 6.0));
    double fac = L.fmax;   // err = 0: grow by the current cap
    if (err2_in_range(err2)) {
        const double y0 = widen(powf(narrow_rn(err2), -0.1f));
        const double y2 = y0 * y0, y4 = y2 * y2, y10 = (y4 * y4) * y2;
        fac = c.safety * fma(y0 * 0.1, fma(-err2, y10, 1.0), y0);
    } else if (positive(err2)) {
        fac = c.safety * pow(err2, -0.1);
    }
    // err2 <= 1 and |Y|^2 > r^2, both sides >= +0 (or err2 NaN: rejected):
    // compared on the bit patterns
    if ((unsigned long long)__double_as_longlong(err2) <= 0x3FF0000000000000ull) {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            L.y[i] = Y[i];
            L.K1[i] = K7[i];
        }
        L.t = last ? c.t_max : L.t + hs;
        ++L.steps;
        L.dm = max_abs(L.dm, D);
        L.h = hs * min_pos(L.fmax, max_pos(c.fac_min, fac));
        L.fmax = c.fac_max;
        if (c.r2 > 0.0 && __double_as_longlong(norm2_fixed(Y)) > __double_as_longlong(c.r2)) L.status = GF_RAY_EXITED;
    } else {
        ++L.rejects;
        L.h = hs * min_pos(L.fmax, max_pos(c.fac_min, fac));
        L.fmax = 1.0;
    }
}

// ------------------------------------------------------- one launch per medium

// The exponential table of the evaluator: 2^(j/2048) as float pairs (DF) or in FP64.
template <bool DF>
__device__ __forceinline__ Tabs stage_tables(double *sT, float *sdT)
{
    if constexpr (DF)
        stage_dfexp_table(sdT);
    else
        stage_exp_table(sT);
    return Tabs{sT, sdT};
}

template <int KIND, bool DF>
__global__ void __launch_bounds__(128) dopri5_medium_kernel(const BatchView B, const int med,
                                                            const int64_t lo, const int64_t hi,
                                                            const RaysView<double> r, int32_t *rejects,
                                                            const Ctl c)
{
    __shared__ double sT[DF ? 1 : kExpTabN];
    __shared__ float sdT[DF ? 2 * kDfExpN : 1];
    // every ray of the launch is in medium `med`: its rows are staged once per block
    __shared__ double srows[DF ? 1 : GF_MAX_BATCH_BLOBS * kBlobStride];
    __shared__ float sprer[DF ? 1 : GF_MAX_BATCH_BLOBS * 4];
    __shared__ float sdfr[DF ? GF_MAX_BATCH_BLOBS * kDfBlobStride : 1];
    const Tabs tb = stage_tables<DF>(sT, sdT);
    const int nbm = B.nb[med];
    if constexpr (DF) {
        for (int j = threadIdx.x; j < nbm * kDfBlobStride; j += blockDim.x)
            sdfr[j] = B.df[(int64_t)med * B.nb_max * kDfBlobStride + j];
    } else {
        for (int j = threadIdx.x; j < nbm * kBlobStride; j += blockDim.x)
            srows[j] = B.blobs[(int64_t)med * B.nb_max * kBlobStride + j];
        if (B.pre != nullptr)
            for (int j = threadIdx.x; j < nbm * 4; j += blockDim.x) sprer[j] = B.pre[(int64_t)med * B.nb_max * 4 + j];
    }
    __syncthreads();
    const int64_t ray = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= hi) return;
    Lane L;
    if (!lane_load<KIND, DF>(L, B, r, med, ray, tb, c)) return;
    // the same values, read from shared memory
    if constexpr (DF) {
        L.dfr = sdfr;
    } else {
        L.rows = srows;
        if (L.prer != nullptr) L.prer = sprer;
    }
    const CoopWarp none{nullptr, nullptr};
    while (L.status == GF_RAY_ACTIVE) lane_attempt<KIND, DF, false>(L, true, tb, c, none);
    lane_store<KIND, DF>(L, r, rejects, tb, c);
}

// ------------------------------------------------------------- persistent

// Warps pop work items (a range of rays of one medium) from a global counter.
// Every `compaction` attempted steps the warp ballots its finished lanes and
// refills them with the next rays of its current item, popping new items as
// items run dry; lanes may hold rays of different media (each lane has its own
// blob slot in shared memory).  RPT ray slots per thread are interleaved.
template <int KIND, int RPT, bool DF>
__global__ void __maxnreg__(168) dopri5_persistent_kernel(const BatchView B, const RaysView<double> r,
                                         int32_t *rejects, const Ctl c,
                                         const int compaction, int *__restrict__ head)
{
    // FP64 blob sums are warp-cooperative (coop_blob_sums, its buffers in
    // dynamic shared memory); the double-float ones run lane by lane on the
    // FP32 pipes, where a lane idle in a divergent term costs little
    constexpr bool kCoop = !DF;
    extern __shared__ double sm_dyn[];
    __shared__ double sT[DF ? 1 : kExpTabN];
    __shared__ float sdT[DF ? 2 * kDfExpN : 1];
    const Tabs tb = stage_tables<DF>(sT, sdT);
    __syncthreads();
    const CoopWarp cw = kCoop ? coop_warp(sm_dyn, B.nb_max) : CoopWarp{nullptr, nullptr};
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    Lane L[RPT];
    bool active[RPT];
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
        active[s] = false;
        // a lane without a ray still runs the cooperative attempts (as a non-participant)
#pragma unroll
        for (int i = 0; i < 6; ++i) L[s].y[i] = L[s].K1[i] = 0.0;
        L[s].h = L[s].t = 0.0;
        L[s].nb = 0;
        L[s].rows = B.blobs;
        L[s].prer = nullptr;
        L[s].dfr = nullptr;
        L[s].mp.kind = KIND;
        L[s].mp.n_h2 = L[s].mp.n02 = L[s].mp.n02a2 = 1.0;
    }
    int64_t cur = 0, end = 0;
    int cur_med = 0;
    bool exhausted = false;
    for (;;) {
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
            unsigned freem = __ballot_sync(0xffffffffu, !active[s]);
            while (freem != 0u && !exhausted) {
                if (cur >= end) {
                    int item = 0;
                    if (lane == 0) item = atomicAdd(head, 1);
                    item = __shfl_sync(0xffffffffu, item, 0);
                    if (item >= B.n_items) {
                        exhausted = true;
                        break;
                    }
                    cur = B.item_begin[item];
                    end = B.item_end[item];
                    cur_med = B.item_medium[item];
                }
                const int nfree = __popc(freem);
                const int take = (int)min((int64_t)nfree, end - cur);
                const int rank = __popc(freem & lt_mask);
                if (!active[s] && rank < take) {
                    if (lane_load<KIND, DF>(L[s], B, r, cur_med, cur + rank, tb, c)) {
                        if (L[s].status == GF_RAY_ACTIVE)
                            active[s] = true;
                        else
                            lane_store<KIND, DF>(L[s], r, rejects, tb, c);
                    }
                }
                cur += take;
                freem = __ballot_sync(0xffffffffu, !active[s]);
            }
        }
        bool any = false;
#pragma unroll
        for (int s = 0; s < RPT; ++s) any = any || active[s];
        if (!__any_sync(0xffffffffu, any)) break;
        for (int it = 0; it < compaction; ++it) {
#pragma unroll
            for (int s = 0; s < RPT; ++s) {
                if constexpr (kCoop) {
                    if (!__any_sync(0xffffffffu, active[s])) continue;   // warp-uniform
                    lane_attempt<KIND, DF, true>(L[s], active[s], tb, c, cw);
                } else if (active[s]) {
                    lane_attempt<KIND, DF, false>(L[s], true, tb, c, cw);
                }
                if (active[s] && L[s].status != GF_RAY_ACTIVE) {
                    lane_store<KIND, DF>(L[s], r, rejects, tb, c);
                    active[s] = false;
                }
            }
        }
    }
}

}  // namespace gf

// ------------------------------------------------------------------- host side

using namespace gf;

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    std::string key;
};

struct gf_batch_s {
    int device = -1;
    int kind = 0, n_media = 0, nb_max = 0;
    std::vector<int64_t> offsets;
    double *d_blobs = nullptr, *d_base = nullptr;
    float *d_pre = nullptr, *d_pre_lim = nullptr, *d_df = nullptr;
    int32_t *d_nb = nullptr;
    gf_precision prec = GF_F64;   // GF_F64 or GF_F64X (gf_batch_set_precision)
    int *d_head = nullptr;
    // work items for the current chunk size
    int chunk = 0, n_items = 0;
    int32_t *d_item_medium = nullptr;
    int64_t *d_item_begin = nullptr, *d_item_end = nullptr;
    cudaStream_t capture = nullptr;
    GraphCache graphs[2];
    bool tuned = false;
    gf_tune tune{};
};

namespace gf {
const double *medium_device_blobs(gf_medium m);
}

static void batch_free(gf_batch b)
{
    dev_free(b->d_blobs);
    dev_free(b->d_pre);
    dev_free(b->d_pre_lim);
    dev_free(b->d_df);
    dev_free(b->d_base);
    dev_free(b->d_nb);
    dev_free(b->d_head);
    dev_free(b->d_item_medium);
    dev_free(b->d_item_begin);
    dev_free(b->d_item_end);
    for (auto &g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
}

static gf_status build_items(gf_batch b, int chunk)
{
    if (b->chunk == chunk && b->d_item_medium) return GF_OK;
    std::vector<int32_t> med;
    std::vector<int64_t> beg, end;
    for (int m = 0; m < b->n_media; ++m)
        for (int64_t lo = b->offsets[m]; lo < b->offsets[m + 1]; lo += chunk) {
            med.push_back(m);
            beg.push_back(lo);
            end.push_back(std::min(lo + chunk, b->offsets[m + 1]));
        }
    dev_free(b->d_item_medium);
    dev_free(b->d_item_begin);
    dev_free(b->d_item_end);
    b->d_item_medium = nullptr;
    b->d_item_begin = b->d_item_end = nullptr;
    b->chunk = 0;   // no valid item list until the rebuild below completes
    b->n_items = 0;
    size_t n = std::max<size_t>(med.size(), 1);
    gf_status s;
    if ((s = cuda_status(dev_alloc(&b->d_item_medium, n * sizeof(int32_t)), "cudaMalloc(items)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&b->d_item_begin, n * sizeof(int64_t)), "cudaMalloc(items)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&b->d_item_end, n * sizeof(int64_t)), "cudaMalloc(items)")) != GF_OK)
        return s;
    if (!med.empty()) {
        cudaMemcpy(b->d_item_medium, med.data(), med.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(b->d_item_begin, beg.data(), beg.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
        if ((s = cuda_status(cudaMemcpy(b->d_item_end, end.data(), end.size() * sizeof(int64_t),
                                        cudaMemcpyHostToDevice), "cudaMemcpy(items)")) != GF_OK)
            return s;
    }
    b->chunk = chunk;
    b->n_items = (int)med.size();
    for (auto &g : b->graphs) g.key.clear();
    return GF_OK;
}

// Device view of a batch; pre = false leaves the pre-test tables out (the
// kernels then decide every blob term in FP64), df adds the double-float rows.
static BatchView view_of(gf_batch b, bool pre, bool df)
{
    BatchView v{};   // fields by name: the kernels trust every pointer they read
    v.n_media = b->n_media;
    v.nb_max = b->nb_max;
    v.n_items = b->n_items;
    v.blobs = b->d_blobs;
    v.pre = pre ? b->d_pre : nullptr;
    v.pre_lim = pre ? b->d_pre_lim : nullptr;
    v.df = df ? b->d_df : nullptr;
    v.nb = b->d_nb;
    v.base = b->d_base;
    v.item_medium = b->d_item_medium;
    v.item_begin = b->d_item_begin;
    v.item_end = b->d_item_end;
    return v;
}

// Every table a launch reads must exist (a view over missing tables would
// make the kernels read through null pointers).
static bool view_complete(gf_batch b, bool pre, bool df, gf_schedule sched)
{
    return b->d_blobs && b->d_nb && b->d_base && (!pre || (b->d_pre && b->d_pre_lim)) && (!df || b->d_df) &&
           (sched != GF_SCHED_PERSISTENT || (b->d_head && b->d_item_medium && b->d_item_begin && b->d_item_end));
}

static Ctl ctl_of(const gf_step_ctl *c, double omega)
{
    Ctl k;
    k.om = make_omega<double>(omega);
    k.rtol = c->rtol;
    k.atol = c->atol;
    k.h0 = c->h0;
    k.t_max = c->t_max;
    k.r2 = c->radius > 0 ? c->radius * c->radius : 0.0;
    k.fac_min = c->fac_min;
    k.fac_max = c->fac_max;
    k.safety = c->safety;
    k.max_steps = c->max_steps;
    // rejections shrink h geometrically to h_min, so attempts are bounded; this
    // cap only guards against a controller that never converges
    k.max_attempts = 4 * c->max_steps + 100000;
    return k;
}

static gf_status check_ctl(const gf_step_ctl *c)
{
    if (c == nullptr || !(c->rtol > 0) || !(c->atol > 0) || !(c->h0 > 0) || !std::isfinite(c->t_max) ||
        !std::isfinite(c->radius) || !(c->fac_min > 0 && c->fac_min < 1) || !(c->fac_max > 1) ||
        !std::isfinite(c->fac_max) || !(c->safety > 0 && c->safety <= 1) || c->max_steps <= 0 ||
        c->max_steps > INT32_MAX / 8) {
        set_error("gf_step_ctl: need rtol, atol, h0 > 0, 0 < fac_min < 1 < fac_max, 0 < safety <= 1, "
                  "finite t_max and radius, 0 < max_steps < 2^28");
        return GF_ERR_INVALID_ARG;
    }
    return GF_OK;
}

static gf_status check_tune(const gf_tune *t)
{
    if (!(t->block == 64 || t->block == 128 || t->block == 256) ||
        !(t->rays_per_thread == 1 || t->rays_per_thread == 2) || t->compaction < 1 ||
        t->compaction > 1024 || t->chunk < 1) {
        set_error("gf_tune: block in {64,128,256}, rays_per_thread in {1,2}, 1 <= compaction <= 1024, chunk >= 1");
        return GF_ERR_INVALID_ARG;
    }
    return GF_OK;
}

static const gf_tune kDefaultTune = {128, 1, 4, 64};

// Launch shape resolved outside any stream capture (function attributes and
// occupancy queries are not stream work).  The kernels read each lane's blob
// rows in place, so a launch needs no dynamic shared memory.
struct LaunchPlan {
    int grid = 0, block = 128, rpt = 1;
    size_t smem = 0;
    bool pre = true;   // FP32 pre-test rows are read (FP64 blob sums)
    bool df = false;   // double-float blob sums (GF_F64X)
};

static void size_slots(gf_batch b, int lanes, LaunchPlan &p, bool persistent)
{
    p.df = b->prec == GF_F64X;
    p.pre = !p.df;
    // the persistent FP64 kernel's cooperative buffers, one set per warp
    p.smem = persistent && !p.df ? (size_t)(lanes / 32) * coop_warp_bytes(b->nb_max) : 0;
}

template <int KIND, int RPT, bool DF>
static cudaError_t plan_persistent_rpt(gf_batch b, const gf_tune &t, LaunchPlan &p)
{
    auto k = dopri5_persistent_kernel<KIND, RPT, DF>;
    p.block = t.block;
    p.rpt = RPT;
    size_slots(b, t.block, p, true);
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, t.block, p.smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    p.grid = sms * per_sm;
    return cudaSuccess;
}

template <int KIND>
static cudaError_t plan(gf_batch b, gf_schedule sched, const gf_tune &t, LaunchPlan &p)
{
    const bool df = b->prec == GF_F64X;
    if (sched == GF_SCHED_PERSISTENT) {
        if (df)
            return t.rays_per_thread == 1 ? plan_persistent_rpt<KIND, 1, true>(b, t, p)
                                          : plan_persistent_rpt<KIND, 2, true>(b, t, p);
        return t.rays_per_thread == 1 ? plan_persistent_rpt<KIND, 1, false>(b, t, p)
                                      : plan_persistent_rpt<KIND, 2, false>(b, t, p);
    }
    p.block = 128;
    size_slots(b, p.block, p, false);
    return df ? cudaFuncSetAttribute(dopri5_medium_kernel<KIND, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)p.smem)
              : cudaFuncSetAttribute(dopri5_medium_kernel<KIND, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)p.smem);
}

template <int KIND>
static cudaError_t launch(gf_batch b, gf_schedule sched, const gf_tune &t, const LaunchPlan &p,
                          const RaysView<double> &r, int32_t *rejects, double omega, const Ctl &c,
                          cudaStream_t s)
{
    const BatchView B = view_of(b, p.pre, p.df);
    if (sched == GF_SCHED_PERSISTENT) {
        cudaError_t e = cudaMemsetAsync(b->d_head, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
#define GF_D5_PERSIST(RPT, DF)                                                                            \
    dopri5_persistent_kernel<KIND, RPT, DF><<<p.grid, p.block, p.smem, s>>>(B, r, rejects, c, t.compaction, \
                                                                          b->d_head)
        if (p.df) {
            if (p.rpt == 1) GF_D5_PERSIST(1, true); else GF_D5_PERSIST(2, true);
        } else {
            if (p.rpt == 1) GF_D5_PERSIST(1, false); else GF_D5_PERSIST(2, false);
        }
#undef GF_D5_PERSIST
        return cudaGetLastError();
    }
    for (int m = 0; m < b->n_media; ++m) {
        const int64_t lo = b->offsets[m], hi = b->offsets[m + 1];
        if (hi <= lo) continue;
        const unsigned blocks = (unsigned)((hi - lo + p.block - 1) / p.block);
        if (p.df)
            dopri5_medium_kernel<KIND, true><<<blocks, p.block, p.smem, s>>>(B, m, lo, hi, r, rejects, c);
        else
            dopri5_medium_kernel<KIND, false><<<blocks, p.block, p.smem, s>>>(B, m, lo, hi, r, rejects, c);
    }
    return cudaGetLastError();
}

#define GF_D5_DISPATCH(FN, ...)                          \
    switch (b->kind) {                                   \
    case K_HOMOG: return FN<K_HOMOG>(__VA_ARGS__);       \
    case K_LUNEBURG: return FN<K_LUNEBURG>(__VA_ARGS__); \
    case K_GRIN: return FN<K_GRIN>(__VA_ARGS__);         \
    case K_QUADRATIC: return FN<K_QUADRATIC>(__VA_ARGS__); \
    default: return cudaErrorInvalidValue;               \
    }

static cudaError_t plan_any(gf_batch b, gf_schedule sched, const gf_tune &t, LaunchPlan &p)
{
    GF_D5_DISPATCH(plan, b, sched, t, p)
}

static cudaError_t enqueue(gf_batch b, gf_schedule sched, const gf_tune &t, const LaunchPlan &p,
                           const RaysView<double> &r, int32_t *rejects, double omega, const Ctl &c,
                           cudaStream_t s)
{
    GF_D5_DISPATCH(launch, b, sched, t, p, r, rejects, omega, c, s)
}

static std::string graph_key(gf_precision prec, gf_schedule sched, const gf_tune &t, const gf_rays *rays,
                             int32_t *rejects, double omega, const gf_step_ctl *c)
{
    char buf[512];
    snprintf(buf, sizeof buf, "p%d|%d|%d,%d,%d,%d|%lld,%lld,%p,%p,%p,%p,%p,%p,%p|%p|%.17g|%.17g,%.17g,%.17g,%.17g,%.17g,%.17g,%.17g,%.17g,%lld",
             (int)prec, (int)sched, t.block, t.rays_per_thread, t.compaction, t.chunk, (long long)rays->n,
             (long long)rays->ld, rays->y, (void *)rays->t, (void *)rays->status, (void *)rays->steps,
             (void *)rays->d_res, (void *)rays->d_max, (void *)rejects, (void *)rejects, omega, c->rtol,
             c->atol, c->h0, c->t_max, c->radius, c->fac_min, c->fac_max, c->safety,
             (long long)c->max_steps);
    return buf;
}

static gf_status run_dopri5(gf_batch b, const gf_rays *rays, int32_t *rejects, double omega,
                            const gf_step_ctl *ctl, gf_schedule sched, const gf_tune &t,
                            cudaStream_t stream, bool use_graph)
{
    gf_status s;
    if (sched == GF_SCHED_PERSISTENT && (s = build_items(b, t.chunk)) != GF_OK) return s;
    const RaysView<double> r{rays->n, rays->ld, (double *)rays->y, rays->t, rays->status, rays->steps,
                             rays->d_res, rays->d_max};
    const Ctl c = ctl_of(ctl, omega);
    LaunchPlan p;
    if ((s = cuda_status(plan_any(b, sched, t, p), "gf_trace_dopri5 launch plan")) != GF_OK) return s;
    if (!view_complete(b, p.pre, p.df, sched)) {
        set_error("gf_trace_dopri5: batch tables missing");
        return GF_ERR_INVALID_ARG;
    }
    if (!use_graph)
        return cuda_status(enqueue(b, sched, t, p, r, rejects, omega, c, stream), "gf_trace_dopri5 launch");
    GraphCache &g = b->graphs[sched];
    const std::string key = graph_key(b->prec, sched, t, rays, rejects, omega, ctl);
    if (g.exec == nullptr || g.key != key) {
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        if (b->capture == nullptr &&
            (s = cuda_status(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking),
                             "cudaStreamCreate")) != GF_OK)
            return s;
        cudaGraph_t graph = nullptr;
        // a capture once begun is always ended before any status is checked, so
        // that no error path can leave the stream (and this thread) capturing
        const cudaError_t be = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        if (be != cudaSuccess) return cuda_status(be, "cudaStreamBeginCapture");
        const cudaError_t le = enqueue(b, sched, t, p, r, rejects, omega, c, b->capture);
        const cudaError_t ce = cudaStreamEndCapture(b->capture, &graph);
        if ((s = cuda_status(le, "gf_trace_dopri5 capture")) != GF_OK ||
            (s = cuda_status(ce, "cudaStreamEndCapture")) != GF_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if ((s = cuda_status(ie, "cudaGraphInstantiate")) != GF_OK) return s;
        g.key = key;
    }
    return cuda_status(cudaGraphLaunch(g.exec, stream), "cudaGraphLaunch");
}

static gf_status check_batch_rays(gf_batch b, const gf_rays *rays, int32_t *rejects)
{
    gf_status s;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != b->device) {
        set_error("batch lives on device %d, current device is %d", b->device, dev);
        return GF_ERR_INVALID_ARG;
    }
    if ((s = check_rays(rays, true)) != GF_OK) return s;
    if (rays->n < b->offsets.back()) {
        set_error("gf_trace_dopri5: rays.n = %lld < offsets[n_media] = %lld", (long long)rays->n,
                  (long long)b->offsets.back());
        return GF_ERR_INVALID_ARG;
    }
    if (rejects && rays->n > 0 && (s = check_device_ptr(rejects, "rejects")) != GF_OK) return s;
    return GF_OK;
}

// ---------------------------------------------------------------- autotune

static std::string tune_key(gf_batch b, const gf_step_ctl *c)
{
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, b->device);
    char buf[400];
    snprintf(buf, sizeof buf, "%s|sm%d|kind%d|nb%d|%s|rtol%.3g|atol%.3g", p.name, p.multiProcessorCount,
             b->kind, b->nb_max, b->prec == GF_F64X ? "f64x" : "f64", c->rtol, c->atol);
    return buf;
}

static bool cache_lookup(const char *path, const std::string &key, gf_tune *out)
{
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        // line format: <key>\t<block> <rpt> <compaction> <chunk>
        char *tab = strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        gf_tune t;
        if (key == line && sscanf(tab + 1, "%d %d %d %d", &t.block, &t.rays_per_thread, &t.compaction,
                                  &t.chunk) == 4 && check_tune(&t) == GF_OK) {
            *out = t;
            found = true;
        }
    }
    fclose(f);
    return found;
}

static void cache_store(const char *path, const std::string &key, const gf_tune &t)
{
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s\t%d %d %d %d\n", key.c_str(), t.block, t.rays_per_thread, t.compaction, t.chunk);
    fclose(f);
}

extern "C" {

gf_status gf_batch_create(const gf_medium *media, int32_t n_media, const int64_t *offsets, gf_batch *out)
{
    if (out == nullptr || media == nullptr || offsets == nullptr || n_media < 1) {
        set_error("gf_batch_create: need media, n_media >= 1, offsets and out");
        return GF_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int dev = -1;
    cudaGetDevice(&dev);
    int kind = -1, nb_max = 0;
    for (int m = 0; m < n_media; ++m) {
        if (media[m] == nullptr || device_of(media[m]) != dev) {
            set_error("gf_batch_create: medium %d is NULL or on another device", m);
            return GF_ERR_INVALID_ARG;
        }
        const MediumParams &p = params_of(media[m]);
        if (p.kind == K_SPLINE || p.kind == K_COLD || (kind >= 0 && p.kind != kind)) {
            set_error("gf_batch_create: media must be isotropic and of one kind (medium %d)", m);
            return GF_ERR_INVALID_ARG;
        }
        if (p.n_blobs > GF_MAX_BATCH_BLOBS) {
            set_error("gf_batch_create: medium %d has %d blobs > %d", m, p.n_blobs, GF_MAX_BATCH_BLOBS);
            return GF_ERR_INVALID_ARG;
        }
        kind = p.kind;
        nb_max = std::max(nb_max, (int)p.n_blobs);
        if (offsets[m] < 0 || offsets[m + 1] < offsets[m]) {
            set_error("gf_batch_create: offsets must be >= 0 and non-decreasing (at %d)", m);
            return GF_ERR_INVALID_ARG;
        }
    }
    gf_batch b = new gf_batch_s();
    b->device = dev;
    b->kind = kind;
    b->n_media = n_media;
    b->nb_max = std::max(nb_max, 1);
    b->offsets.assign(offsets, offsets + n_media + 1);
    std::vector<double> base(3 * (size_t)n_media);
    std::vector<float> pre_lim(n_media);
    std::vector<int32_t> nb(n_media);
    gf_status s = GF_OK;
    const size_t row = (size_t)b->nb_max * kBlobStride, prow = (size_t)b->nb_max * 4,
                 drow = (size_t)b->nb_max * kDfBlobStride;
    if ((s = cuda_status(dev_alloc(&b->d_blobs, row * n_media * sizeof(double)), "cudaMalloc(batch)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&b->d_df, drow * n_media * sizeof(float)), "cudaMalloc(batch)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&b->d_pre, prow * n_media * sizeof(float)), "cudaMalloc(batch)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&b->d_pre_lim, pre_lim.size() * sizeof(float)), "cudaMalloc(batch)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&b->d_base, base.size() * sizeof(double)), "cudaMalloc(batch)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&b->d_nb, nb.size() * sizeof(int32_t)), "cudaMalloc(batch)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&b->d_head, sizeof(int)), "cudaMalloc(batch)")) != GF_OK) {
        batch_free(b);
        return s;
    }
    for (int m = 0; m < n_media; ++m) {
        const MediumParams &p = params_of(media[m]);
        base[3 * m] = p.n_h2;
        base[3 * m + 1] = p.n02;
        base[3 * m + 2] = p.n02a2;
        pre_lim[m] = p.pre_lim;
        nb[m] = p.n_blobs;
        if (p.n_blobs > 0 &&
            ((s = cuda_status(cudaMemcpy(b->d_blobs + row * m, medium_device_blobs(media[m]),
                                         p.n_blobs * kBlobStride * sizeof(double), cudaMemcpyDeviceToDevice),
                              "cudaMemcpy(batch blobs)")) != GF_OK ||
             (s = cuda_status(cudaMemcpy(b->d_pre + prow * m, p.pre32, p.n_blobs * 4 * sizeof(float),
                                         cudaMemcpyDeviceToDevice), "cudaMemcpy(batch blobs)")) != GF_OK ||
             (s = cuda_status(cudaMemcpy(b->d_df + drow * m, p.dfrows, p.n_blobs * kDfBlobStride * sizeof(float),
                                         cudaMemcpyDeviceToDevice), "cudaMemcpy(batch blobs)")) != GF_OK)) {
            batch_free(b);
            return s;
        }
    }
    if ((s = cuda_status(cudaMemcpy(b->d_base, base.data(), base.size() * sizeof(double),
                                    cudaMemcpyHostToDevice), "cudaMemcpy(batch)")) != GF_OK ||
        (s = cuda_status(cudaMemcpy(b->d_pre_lim, pre_lim.data(), pre_lim.size() * sizeof(float),
                                    cudaMemcpyHostToDevice), "cudaMemcpy(batch)")) != GF_OK ||
        (s = cuda_status(cudaMemcpy(b->d_nb, nb.data(), nb.size() * sizeof(int32_t), cudaMemcpyHostToDevice),
                         "cudaMemcpy(batch)")) != GF_OK) {
        batch_free(b);
        return s;
    }
    *out = b;
    return GF_OK;
}

gf_status gf_batch_set_precision(gf_batch b, gf_precision prec)
{
    if (b == nullptr) {
        set_error("gf_batch_set_precision: batch is NULL");
        return GF_ERR_INVALID_ARG;
    }
    if (prec != GF_F64 && prec != GF_F64X) {
        set_error("gf_batch_set_precision: DOPRI5 runs in GF_F64 or GF_F64X");
        return GF_ERR_UNSUPPORTED;
    }
    if (prec != b->prec) {
        b->prec = prec;
        b->tuned = false;   // a launch shape tuned for the other mode
    }
    return GF_OK;
}

gf_status gf_batch_destroy(gf_batch b)
{
    if (b == nullptr) return GF_OK;
    cudaDeviceSynchronize();
    batch_free(b);
    return GF_OK;
}

gf_status gf_trace_dopri5(gf_batch b, const gf_rays *rays, int32_t *rejects, double omega,
                          const gf_step_ctl *ctl, gf_schedule sched, const gf_tune *tune, void *stream)
{
    gf_status s;
    if (b == nullptr) {
        set_error("gf_trace_dopri5: batch is NULL");
        return GF_ERR_INVALID_ARG;
    }
    if (sched != GF_SCHED_PERSISTENT && sched != GF_SCHED_PER_MEDIUM) {
        set_error("gf_trace_dopri5: unknown schedule %d", (int)sched);
        return GF_ERR_INVALID_ARG;
    }
    if (!(omega > 0) || !std::isfinite(omega)) {
        set_error("gf_trace_dopri5: omega must be positive and finite");
        return GF_ERR_INVALID_ARG;
    }
    if ((s = check_ctl(ctl)) != GF_OK) return s;
    if ((s = check_batch_rays(b, rays, rejects)) != GF_OK) return s;
    const gf_tune t = tune ? *tune : (b->tuned ? b->tune : kDefaultTune);
    if ((s = check_tune(&t)) != GF_OK) return s;
    if (rays->n == 0 || b->offsets.back() == b->offsets.front()) return GF_OK;
    return run_dopri5(b, rays, rejects, omega, ctl, sched, t, (cudaStream_t)stream, true);
}

gf_status gf_dopri5_autotune(gf_batch b, const gf_rays *rays, double omega, const gf_step_ctl *ctl,
                             const char *cache_path, gf_tune *out)
{
    gf_status s;
    if (b == nullptr || out == nullptr) {
        set_error("gf_dopri5_autotune: batch and out must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    if ((s = check_ctl(ctl)) != GF_OK) return s;
    if ((s = check_batch_rays(b, rays, nullptr)) != GF_OK) return s;
    const std::string key = tune_key(b, ctl);
    if (cache_lookup(cache_path, key, out)) {
        b->tune = *out;
        b->tuned = true;
        return GF_OK;
    }
    // prefix of media holding ~1/8 of the rays (>= 65,536 when available)
    const int64_t total = b->offsets.back() - b->offsets.front();
    const int64_t want = std::max<int64_t>(total / 8, std::min<int64_t>(total, 65536));
    int m_end = 0;
    while (m_end < b->n_media && b->offsets[m_end + 1] - b->offsets.front() < want) ++m_end;
    m_end = std::min(b->n_media, m_end + 1);
    const int64_t lo = b->offsets.front(), hi = b->offsets[m_end], n = hi - lo;
    // scratch copies of the sample rays
    double *y = nullptr, *t = nullptr, *dres = nullptr, *dmax = nullptr;
    int32_t *st = nullptr, *steps = nullptr;
    auto release = [&]() {
        dev_free(y); dev_free(t); dev_free(dres); dev_free(dmax); dev_free(st); dev_free(steps);
    };
    if ((s = cuda_status(dev_alloc(&y, 6 * n * sizeof(double)), "cudaMalloc(tune)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&t, n * sizeof(double)), "cudaMalloc(tune)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&dres, n * sizeof(double)), "cudaMalloc(tune)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&dmax, n * sizeof(double)), "cudaMalloc(tune)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&st, n * sizeof(int32_t)), "cudaMalloc(tune)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&steps, n * sizeof(int32_t)), "cudaMalloc(tune)")) != GF_OK) {
        release();
        return s;
    }
    // a sub-batch view over media [0, m_end) with offsets shifted to the scratch rays
    gf_batch_s sub;
    sub.device = b->device;
    sub.kind = b->kind;
    sub.n_media = m_end;
    sub.nb_max = b->nb_max;
    sub.offsets.assign(b->offsets.begin(), b->offsets.begin() + m_end + 1);
    for (auto &o : sub.offsets) o -= lo;
    sub.d_blobs = b->d_blobs;
    sub.d_pre = b->d_pre;
    sub.d_pre_lim = b->d_pre_lim;
    sub.d_df = b->d_df;
    sub.prec = b->prec;
    sub.d_base = b->d_base;
    sub.d_nb = b->d_nb;
    if ((s = cuda_status(dev_alloc(&sub.d_head, sizeof(int)), "cudaMalloc(tune)")) != GF_OK) {
        dev_free(sub.d_head);   // allocated when only the status check failed
        release();
        return s;
    }
    const gf_rays scratch{n, n, y, t, st, steps, dres, dmax};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const double *src_y = (const double *)rays->y;
    auto reset = [&]() {
        for (int c = 0; c < 6; ++c)
            cudaMemcpy(y + c * n, src_y + c * rays->ld + lo, n * sizeof(double), cudaMemcpyDeviceToDevice);
        cudaMemcpy(t, rays->t + lo, n * sizeof(double), cudaMemcpyDeviceToDevice);
        cudaMemcpy(st, rays->status + lo, n * sizeof(int32_t), cudaMemcpyDeviceToDevice);
        cudaMemcpy(steps, rays->steps + lo, n * sizeof(int32_t), cudaMemcpyDeviceToDevice);
        cudaMemset(dmax, 0, n * sizeof(double));
    };
    static const int blocks[] = {64, 128, 256};
    static const int rpts[] = {1, 2};
    static const int comps[] = {1, 4, 16};
    static const int chunks[] = {32, 256};
    gf_tune best = kDefaultTune;
    float best_ms = 1e30f;
    for (int bl : blocks)
        for (int rp : rpts)
            for (int cp : comps)
                for (int ch : chunks) {
                    gf_tune cand{bl, rp, cp, ch};
                    reset();
                    cudaEventRecord(e0);
                    gf_status rs = run_dopri5(&sub, &scratch, nullptr, omega, ctl, GF_SCHED_PERSISTENT,
                                              cand, nullptr, false);
                    cudaEventRecord(e1);
                    cudaError_t se = cudaEventSynchronize(e1);
                    if (rs != GF_OK || se != cudaSuccess) {
                        cudaGetLastError();
                        continue;  // e.g. a shape that does not fit; try the next
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = cand;
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(sub.d_head);
    dev_free(sub.d_item_medium);
    dev_free(sub.d_item_begin);
    dev_free(sub.d_item_end);
    sub.d_blobs = nullptr;
    sub.d_pre = sub.d_pre_lim = sub.d_df = nullptr;
    sub.d_base = nullptr;
    sub.d_nb = nullptr;
    sub.d_head = nullptr;
    sub.d_item_medium = nullptr;
    sub.d_item_begin = sub.d_item_end = nullptr;
    release();
    if (best_ms >= 1e29f) {
        set_error("gf_dopri5_autotune: no launch shape ran");
        return GF_ERR_CUDA;
    }
    *out = best;
    b->tune = best;
    b->tuned = true;
    cache_store(cache_path, key, best);
    return GF_OK;
}

}  // extern "C"
