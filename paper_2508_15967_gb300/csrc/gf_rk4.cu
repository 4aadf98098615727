// gf_rk4.cu -- fused fixed-step RK4 ray-tracing kernel and the on-shell
// initialisation kernel.
//
// One thread owns one ray for the whole call: the state is loaded once,
// advanced n_steps times in registers (four fused D / grad D evaluations per
// step) and stored once -- the load-once / store-once kernel shape of the
// paper's generated RK4 ray update (Sec. 2.2, Sec. 4).  The blob table is
// staged in shared memory and read as warp-wide broadcasts.
#include "gf_dfloat.cuh"
#include "gf_internal.cuh"

namespace gf {

// Right-hand side with the blob sums in double-float (GF_F64X): base index,
// D and f in FP64 exactly as rhs_iso, blob terms from blobs_df.
template <int KIND>
struct RhsDF {
    const MediumParams &m;
    int nb;
    Omega<double> om;
    template <bool WANT_D = true>
    __device__ __forceinline__ bool eval(const double *y, double *f, double &D, EvalCtx<double> &cx) const
    {
        return rhs_df<KIND, WANT_D>(m, cx.dfb, nb, 1, om, y, f, D, cx.dfT, cx.live);
    }
};

template <typename R, int KIND, bool DF>
struct RhsSel {
    using type = Rhs<R, KIND>;
    static __device__ __forceinline__ type make(const MediumParams &m, const R *sb, const Omega<R> &om)
    {
        return type{m, sb, m.n_blobs, om};
    }
};
template <int KIND>
struct RhsSel<double, KIND, true> {
    using type = RhsDF<KIND>;
    static __device__ __forceinline__ type make(const MediumParams &m, const double *, const Omega<double> &om)
    {
        return type{m, m.n_blobs, om};
    }
};

constexpr int kRk4Block = 128;

template <typename R>
__device__ __forceinline__ bool finite6(const R *y)
{
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 6; ++c) ok = ok && isfinite(y[c]);
    return ok;
}
// Doubles: exponent field not all ones, tested on the high words (integer pipe).
template <>
__device__ __forceinline__ bool finite6<double>(const double *y)
{
    unsigned bad = 0u;
#pragma unroll
    for (int c = 0; c < 6; ++c) bad |= finite_bits(y[c]) ? 0u : 1u;
    return bad == 0u;
}

// State update y <- y + inc.  FP64: one rounded addition.  FP32: Kahan-compensated
// (Kahan 1965) so that 10^4 small increments to |x| ~ 1 do not drift.
// Components NC..5 have a zero right-hand side and are carried unchanged.
template <typename R>
struct Accum {
    template <int NC>
    __device__ __forceinline__ void add(R *y, const R *inc, R *out) const
    {
#pragma unroll
        for (int c = 0; c < 6; ++c) out[c] = c < NC ? __dadd_rn(y[c], inc[c]) : y[c];
    }
    __device__ __forceinline__ void commit(R *y, const R *out) {
#pragma unroll
        for (int c = 0; c < 6; ++c) y[c] = out[c];
    }
};

template <>
struct Accum<float> {
    float comp[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float pend[6];
    template <int NC>
    __device__ __forceinline__ void add(float *y, const float *inc, float *out)
    {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (c >= NC) {
                pend[c] = comp[c];
                out[c] = y[c];
                continue;
            }
            float yk = __fsub_rn(inc[c], comp[c]);
            float s = __fadd_rn(y[c], yk);
            pend[c] = __fsub_rn(__fsub_rn(s, y[c]), yk);
            out[c] = s;
        }
    }
    __device__ __forceinline__ void commit(float *y, const float *out)
    {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            y[c] = out[c];
            comp[c] = pend[c];
        }
    }
};

// Warp-aggregated add of per-thread work counts (evaluations, blob terms).
__device__ __forceinline__ void add_work(unsigned long long *counters, long long evals, long long terms)
{
    if (counters == nullptr) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        evals += __shfl_down_sync(0xffffffffu, evals, o);
        terms += __shfl_down_sync(0xffffffffu, terms, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(counters, (unsigned long long)evals);
        atomicAdd(counters + 1, (unsigned long long)terms);
    }
}

template <typename R, int KIND, bool DF>
__global__ void __launch_bounds__(kRk4Block, (KIND == K_SPLINE || KIND == K_COLD) ? 1 : sizeof(R) == 4 ? 6 : 5)
rk4_kernel(const MediumParams m, const RaysView<R> r, const Omega<R> om, const R dt, const double dt64,
           const int64_t n_steps, const R radius2, const int64_t every, double *__restrict__ ckpt,
           unsigned long long *counters)
{
    // FP64 blob terms: scaled rows, the FP32 pre-test rows and the exp table
    constexpr bool kBlobs64 = sizeof(R) == 8 && KIND != K_SPLINE && KIND != K_COLD && !DF;
    __shared__ __align__(16) R sb[kBlobStride * GF_MAX_BLOBS];
    __shared__ double sT[kBlobs64 ? kExpTabN : 1];
    __shared__ float sp[kBlobs64 ? 4 * GF_MAX_BLOBS : 1];
    __shared__ float sdf[DF ? kDfBlobStride * GF_MAX_BLOBS : 1];
    __shared__ float sdT[DF ? 2 * kDfExpN : 1];
    if constexpr (KIND != K_SPLINE && !DF) stage_blobs<R>(m, sb);
    if constexpr (kBlobs64) {
        stage_pretest(m, sp);
        stage_exp_table(sT);
    }
    if constexpr (DF) {
        stage_df_blobs(m, sdf);
        stage_dfexp_table(sdT);
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int st = GF_RAY_DONE;   // lanes without an active ray skip the loop
    R y[6];
    R dm = (R)0;
    if (i < r.n) st = r.status[i];
    EvalCtx<R> cx;
    if constexpr (kBlobs64) {
        cx.T = sT;
        cx.pre = sp;
    }
    if constexpr (DF) {
        cx.dfb = sdf;
        cx.dfT = sdT;
    }
    long long evals = 0;
    int64_t s = 0;
    const auto f = RhsSel<R, KIND, DF>::make(m, sb, om);
    if (st == GF_RAY_ACTIVE) {
#pragma unroll
        for (int c = 0; c < 6; ++c) y[c] = r.y[c * r.ld + i];
        dm = r.d_max ? (R)r.d_max[i] : (R)0;
        const R h2 = dt * (R)0.5, h6 = dt / (R)6;
        // the cold plasma's k_y, k_z are constants of motion (f_4 = f_5 = 0):
        // only the first NC components are combined
        constexpr int NC = KIND == K_COLD ? 4 : 6;
        Accum<R> acc_state;
        for (; s < n_steps; ++s) {
            if (ckpt != nullptr && s % every == 0) {
                double *slot = ckpt + (s / every) * 6 * r.n;
#pragma unroll
                for (int c = 0; c < 6; ++c) slot[c * r.n + i] = (double)y[c];
            }
            R K[6], acc[6], Y[6], D;
            evals += 4;
            bool ok = f.template eval<true>(y, K, D, cx);
            dm = max_abs(dm, D);
            if (!ok) { st = GF_RAY_CUTOFF; break; }
#pragma unroll
            for (int c = 0; c < 6; ++c) { acc[c] = K[c]; Y[c] = c < NC ? rk_axpy(h2, K[c], y[c]) : y[c]; }
            if (!f.template eval<false>(Y, K, D, cx)) { st = GF_RAY_CUTOFF; break; }
#pragma unroll
            for (int c = 0; c < NC; ++c) { acc[c] = rk_acc2(acc[c], K[c]); Y[c] = rk_axpy(h2, K[c], y[c]); }
            if (!f.template eval<false>(Y, K, D, cx)) { st = GF_RAY_CUTOFF; break; }
#pragma unroll
            for (int c = 0; c < NC; ++c) { acc[c] = rk_acc2(acc[c], K[c]); Y[c] = rk_axpy(dt, K[c], y[c]); }
            if (!f.template eval<false>(Y, K, D, cx)) { st = GF_RAY_CUTOFF; break; }
            R inc[6], yn[6];
#pragma unroll
            for (int c = 0; c < NC; ++c) inc[c] = rk_inc(h6, acc[c], K[c]);
            acc_state.template add<NC>(y, inc, yn);
            if (!finite6(yn)) { st = GF_RAY_NONFINITE; break; }
            acc_state.commit(y, yn);
            if (radius2 > (R)0 && norm2_fixed(y) > radius2) {
                st = GF_RAY_EXITED;
                ++s;
                break;
            }
        }
        // s = number of steps applied in this call
        R K[6], D;
        f.template eval<true>(y, K, D, cx);
        ++evals;
        dm = max_abs(dm, D);
        if (r.d_res) r.d_res[i] = (double)fabs(D);
        if (r.d_max) r.d_max[i] = (double)dm;
#pragma unroll
        for (int c = 0; c < 6; ++c) r.y[c * r.ld + i] = y[c];
        if (s > 0) r.t[i] = __dadd_rn(r.t[i], __dmul_rn((double)s, dt64));
        r.steps[i] += (int32_t)s;
        r.status[i] = st;
    }
    add_work(counters, evals, cx.live);
}

// ------------------------------------------- small traces: components split

// A trace with few rays leaves most SM sub-partitions idle, and one warp's
// FP64 instruction occupies its sub-partition for ~64 cycles whatever the
// number of its active lanes, so such a trace takes (FP64 instructions of a
// step per warp) x 64 cycles a step, however its rays are spread over warps.
// Here kSplitWarps warps share 32 rays: warp w advances the components c with
// c mod kSplitWarps = w (the stage points, the slope sums and the update of
// those), and every warp evaluates what all components need (index law, blob
// sums, reciprocal of n^2) at the full stage point, which the warps exchange
// through shared memory once per stage.  Each value is formed by the same
// operations as in rk4_kernel, so both kernels return the same bits.  Every
// thread of a block passes the same barriers: the stops are decided from the
// exchanged (identical) values, and the loop ends by a block-wide vote.
// (measured on the 1024-ray Luneburg trace: 1, 2, 3 and 6 warps per 32 rays
// take 9.1, 8.0, 7.0 and 7.5 ms; a 1000-ray GRIN trace with 16 blobs 77.8,
// 72.6, 68.8 and 83.8 ms)
constexpr int kSplitWarps = 3;
static_assert(6 % kSplitWarps == 0, "each warp owns 6 / kSplitWarps components");

template <int KIND, int W>
__device__ __forceinline__ void rk4_split_warp(const MediumParams &m, const RaysView<double> &r,
                                               const Omega<double> &om, const double dt, const double dt64,
                                               const int64_t n_steps, const double radius2, const int64_t every,
                                               double *__restrict__ ckpt, unsigned long long *counters,
                                               const double *sb, EvalCtx<double> &cx, double (*xb)[6][32])
{
    constexpr int NO = 6 / kSplitWarps;   // this warp's components: W + kSplitWarps j, j < NO
    const int lane = (int)(threadIdx.x & 31u);
    const int64_t i = (int64_t)blockIdx.x * 32 + lane;
    int st = GF_RAY_DONE;
    if (i < r.n) st = r.status[i];
    const bool started = st == GF_RAY_ACTIVE;
    bool act = started;
    double y[6], dm = 0.0;
    if (started) {
#pragma unroll
        for (int c = 0; c < 6; ++c) y[c] = r.y[c * r.ld + i];
        dm = r.d_max ? r.d_max[i] : 0.0;
    }
    const Rhs<double, KIND> f{m, sb, m.n_blobs, om};
    const double h2 = dt * 0.5, h6 = dt / 6.0;
    long long evals = 0;
    int64_t s = 0;
    int b = 0;
    // the stage point Y: own components computed, the others read from the exchange
    auto exchange = [&](double *Y, bool live) {
        if (live) {
#pragma unroll
            for (int j = 0; j < NO; ++j) xb[b][W + kSplitWarps * j][lane] = Y[W + kSplitWarps * j];
        }
        __syncthreads();
        if (live) {
#pragma unroll
            for (int c = 0; c < 6; ++c)
                if (c % kSplitWarps != W) Y[c] = xb[b][c][lane];
        }
        b ^= 1;
    };
    for (int64_t it = 0; it < n_steps; ++it) {
        // a block-wide decision, so that every thread of the block passes the same barriers
        if (!__syncthreads_or(act)) break;
        double K[6], Y[6], D, acc[NO];
        if (act) {
            if (ckpt != nullptr && s % every == 0) {
                double *slot = ckpt + (s / every) * 6 * r.n;
#pragma unroll
                for (int j = 0; j < NO; ++j) slot[(W + kSplitWarps * j) * r.n + i] = y[W + kSplitWarps * j];
            }
            evals += 4;
            const bool ok = f.template eval<true>(y, K, D, cx);
            dm = max_abs(dm, D);
            if (!ok) { st = GF_RAY_CUTOFF; act = false; }
        }
        if (act) {
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                const int c = W + kSplitWarps * j;
                acc[j] = K[c];
                Y[c] = rk_axpy(h2, K[c], y[c]);
            }
        }
        exchange(Y, act);
        if (act && !f.template eval<false>(Y, K, D, cx)) { st = GF_RAY_CUTOFF; act = false; }
        if (act) {
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                const int c = W + kSplitWarps * j;
                acc[j] = rk_acc2(acc[j], K[c]);
                Y[c] = rk_axpy(h2, K[c], y[c]);
            }
        }
        exchange(Y, act);
        if (act && !f.template eval<false>(Y, K, D, cx)) { st = GF_RAY_CUTOFF; act = false; }
        if (act) {
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                const int c = W + kSplitWarps * j;
                acc[j] = rk_acc2(acc[j], K[c]);
                Y[c] = rk_axpy(dt, K[c], y[c]);
            }
        }
        exchange(Y, act);
        if (act && !f.template eval<false>(Y, K, D, cx)) { st = GF_RAY_CUTOFF; act = false; }
        double yn[6];
        if (act) {
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                const int c = W + kSplitWarps * j;
                yn[c] = __dadd_rn(y[c], rk_inc(h6, acc[j], K[c]));
            }
        }
        exchange(yn, act);
        if (act) {
            if (!finite6(yn)) {
                st = GF_RAY_NONFINITE;
                act = false;
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) y[c] = yn[c];
                ++s;
                if (radius2 > 0.0 && norm2_fixed(y) > radius2) {
                    st = GF_RAY_EXITED;
                    act = false;
                }
            }
        }
    }
    if (started) {
#pragma unroll
        for (int j = 0; j < NO; ++j) r.y[(W + kSplitWarps * j) * r.ld + i] = y[W + kSplitWarps * j];
        if constexpr (W == 0) {
            double K[6], D;
            f.template eval<true>(y, K, D, cx);
            ++evals;
            dm = max_abs(dm, D);
            if (r.d_res) r.d_res[i] = fabs(D);
            if (r.d_max) r.d_max[i] = dm;
            if (s > 0) r.t[i] = __dadd_rn(r.t[i], __dmul_rn((double)s, dt64));
            r.steps[i] += (int32_t)s;
            r.status[i] = st;
        }
    }
    if constexpr (W == 0) add_work(counters, evals, cx.live);
}

template <int KIND, int W = 0>
__device__ __forceinline__ void rk4_split_dispatch(int w, const MediumParams &m, const RaysView<double> &r,
                                                   const Omega<double> &om, const double dt, const int64_t n_steps,
                                                   const double radius2, const int64_t every, double *ckpt,
                                                   unsigned long long *counters, const double *sb,
                                                   EvalCtx<double> &cx, double (*xb)[6][32])
{
    if constexpr (W < kSplitWarps) {
        if (w == W)
            rk4_split_warp<KIND, W>(m, r, om, dt, dt, n_steps, radius2, every, ckpt, counters, sb, cx, xb);
        else
            rk4_split_dispatch<KIND, W + 1>(w, m, r, om, dt, n_steps, radius2, every, ckpt, counters, sb, cx, xb);
    }
}

template <int KIND>
__global__ void __launch_bounds__(32 * kSplitWarps, 1)
rk4_split_kernel(const MediumParams m, const RaysView<double> r, const Omega<double> om, const double dt,
                 const int64_t n_steps, const double radius2, const int64_t every, double *__restrict__ ckpt,
                 unsigned long long *counters)
{
    __shared__ __align__(16) double sb[kBlobStride * GF_MAX_BLOBS];
    __shared__ double sT[kExpTabN];
    __shared__ float sp[4 * GF_MAX_BLOBS];
    __shared__ double xb[2][6][32];
    stage_blobs<double>(m, sb);
    stage_pretest(m, sp);
    stage_exp_table(sT);
    __syncthreads();
    EvalCtx<double> cx;
    cx.T = sT;
    cx.pre = sp;
    rk4_split_dispatch<KIND>((int)(threadIdx.x >> 5), m, r, om, dt, n_steps, radius2, every, ckpt, counters, sb,
                             cx, xb);
}

// k = s d with D(x, s d, w) = 0, s = w sqrt(eps / q).
template <typename R, int KIND>
__global__ void __launch_bounds__(kRk4Block) onshell_kernel(const MediumParams m, const RaysView<R> r,
                                                            const R *__restrict__ dir, const R omega)
{
    __shared__ __align__(16) R sb[kBlobStride * GF_MAX_BLOBS];
    __shared__ double sT[sizeof(R) == 8 ? kExpTabN : 1];
    if constexpr (KIND != K_SPLINE) stage_blobs<R>(m, sb);
    if constexpr (sizeof(R) == 8) stage_exp_table(sT);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r.n) return;
    R x[3] = {r.y[i], r.y[r.ld + i], r.y[2 * r.ld + i]};
    R d[3] = {dir[i], dir[r.ld + i], dir[2 * r.ld + i]};
    R eps, q;
    if constexpr (KIND == K_SPLINE) {
        R val[7], grad[7][3];
        spline_fields<R>(m, x, val, grad);
        eps = val[6];
        R Md0 = val[0] * d[0] + val[1] * d[1] + val[2] * d[2];
        R Md1 = val[1] * d[0] + val[3] * d[1] + val[4] * d[2];
        R Md2 = val[2] * d[0] + val[4] * d[1] + val[5] * d[2];
        q = d[0] * Md0 + d[1] * Md1 + d[2] * Md2;
    } else {
        R g[3];
        EvalCtx<R> cx;
        cx.T = sT;
        iso_index<R, KIND>(m, sb, m.n_blobs, x, eps, g, cx);
        q = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    }
    if (!(eps > (R)0) || !(q > (R)0)) {
        r.status[i] = GF_RAY_CUTOFF;
        for (int c = 0; c < 3; ++c) r.y[(3 + c) * r.ld + i] = (R)0;
        return;
    }
    R sc = omega * sqrt(eps / q);
    r.status[i] = GF_RAY_ACTIVE;
    for (int c = 0; c < 3; ++c) r.y[(3 + c) * r.ld + i] = sc * d[c];
}

// The paper's ray initialisation (Sec. 4): w, x, k_y, k_z fixed, k_x from
// Newton on D = 0 to |D| < tol, starting from the k_x held in the rays; the
// medium (n^2, or M and eps) is evaluated once at x, after which D is a
// quadratic in k_x and every iteration is a few scalar operations.
template <typename R, int KIND>
__global__ void __launch_bounds__(kRk4Block) newton_kx_kernel(const MediumParams m, const RaysView<R> r,
                                                              const R omega, const R tol, const int max_iter)
{
    __shared__ __align__(16) R sb[kBlobStride * GF_MAX_BLOBS];
    __shared__ double sT[sizeof(R) == 8 ? kExpTabN : 1];
    if constexpr (KIND != K_SPLINE) stage_blobs<R>(m, sb);
    if constexpr (sizeof(R) == 8) stage_exp_table(sT);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r.n) return;
    const R x[3] = {r.y[i], r.y[r.ld + i], r.y[2 * r.ld + i]};
    R kx = r.y[3 * r.ld + i];
    const R ky = r.y[4 * r.ld + i], kz = r.y[5 * r.ld + i];
    if constexpr (KIND == K_COLD) {
        // D is quartic in k_x: full evaluation per iteration (D and dD/dk_x)
        const Omega<R> om = make_omega<R>((double)omega);
        bool ok = false;
        for (int it = 0; it < max_iter; ++it) {
            R yy[6] = {x[0], x[1], x[2], kx, ky, kz}, f[6], D;
            const bool live = rhs_cold<R>(m, om, yy, f, D);
            if (fabs(D) < tol) { ok = true; break; }
            // f_x0 = -D_kx / D_w  and D_w is returned through f: recover D_kx
            if (!live) break;
            R Dkx = cold_dkx<R>(m, om, yy);
            if (Dkx == (R)0 || !isfinite(D)) break;
            const R step = D / Dkx;
            kx = kx - step;
            if (fabs(step) <= (R)0x1p-50 * fabs(kx)) {
                R y2[6] = {x[0], x[1], x[2], kx, ky, kz}, f2[6], D2;
                rhs_cold<R>(m, om, y2, f2, D2);
                ok = fabs(D2) <= (R)8 * tol;
                break;
            }
        }
        r.y[3 * r.ld + i] = kx;
        r.status[i] = ok ? GF_RAY_ACTIVE : GF_RAY_CUTOFF;
        return;
    }
    // D(k_x) = a k_x^2 + 2 b k_x + c  with  dD/dk_x = 2 (a k_x + b)
    R a, b, c;
    if constexpr (KIND == K_SPLINE) {
        R val[7], grad[7][3];
        spline_fields<R>(m, x, val, grad);
        a = val[0];
        b = val[1] * ky + val[2] * kz;
        c = val[3] * ky * ky + (R)2 * val[4] * ky * kz + val[5] * kz * kz - omega * omega * val[6];
    } else {
        R n2, g[3];
        EvalCtx<R> cx;
        cx.T = sT;
        iso_index<R, KIND>(m, sb, m.n_blobs, x, n2, g, cx);
        a = (R)1;
        b = (R)0;
        c = ky * ky + kz * kz - omega * omega * n2;
    }
    bool ok = false;
    for (int it = 0; it < max_iter; ++it) {
        const R D = (a * kx + (R)2 * b) * kx + c;
        if (fabs(D) < tol) { ok = true; break; }
        const R Dk = (R)2 * (a * kx + b);
        if (Dk == (R)0 || !isfinite(D)) break;
        const R step = D / Dk;
        kx = kx - step;
        if (fabs(step) <= (R)0x1p-50 * fabs(kx)) {
            const R D2 = (a * kx + (R)2 * b) * kx + c;
            ok = fabs(D2) <= (R)8 * tol;
            break;
        }
    }
    r.y[3 * r.ld + i] = kx;
    r.status[i] = ok ? GF_RAY_ACTIVE : GF_RAY_CUTOFF;
}

template <typename R>
static RaysView<R> view(const gf_rays &r)
{
    return RaysView<R>{r.n, r.ld, (R *)r.y, r.t, r.status, r.steps, r.d_res, r.d_max};
}

// Threads per block of the RK4 kernel: 128 when the rays fill every SM; a
// launch with fewer rays than SMs x 128 uses warps of its own (32-thread
// blocks), spreading them over up to four times as many SMs -- each ray's
// steps are bound by the FP64 pipe of the SM it runs on.
static int rk4_block_small(int64_t n)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return kRk4Block;
    return n >= (int64_t)sms * kRk4Block ? kRk4Block : 32;
}

// Block size of a launch of kernel k over n rays.  Every ray's steps are
// bound by the FP64 pipe of its SM, so when all blocks are resident at once
// the trace takes as long as the SM holding the most warps: 65,536 rays in
// 512 blocks of 128 on 152 SMs put 4 blocks on some SMs and 3 on others (84%
// of the SMs' time used), in 1,024 blocks of 64 at most 7 against 6.74 on
// average (96%).  Among 128, 64 and 32 the size that keeps one resident wave
// with the best balance is chosen; launches of several waves keep 128.
template <typename K>
static int rk4_block(K kernel, int64_t n)
{
    const int fallback = rk4_block_small(n);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return fallback;
    if (fallback == 32) return 32;
    int best = kRk4Block;
    double best_eff = -1.0;
    for (int b : {kRk4Block, kRk4Block / 2, kRk4Block / 4}) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, b, 0) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            continue;
        }
        const int64_t blocks = (n + b - 1) / b;
        if (blocks > (int64_t)sms * per_sm) {   // more than one wave
            if (b == kRk4Block) return kRk4Block;
            continue;
        }
        const double avg = (double)blocks / sms, max = (double)((blocks + sms - 1) / sms);
        const double eff = avg / max;
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = b;
        }
    }
    return best;
}

template <typename R, int KIND, bool DF = false>
static cudaError_t rk4_launch(const MediumParams &m, const gf_rays &r, double omega, double dt,
                              int64_t n_steps, double radius, int64_t every, double *ckpt,
                              cudaStream_t s)
{
    const R r2 = radius > 0 ? (R)(radius * radius) : (R)0;
    if constexpr (sizeof(R) == 8 && !DF && KIND != K_SPLINE && KIND != K_COLD) {
        // few rays: three warps per 32 rays while they fit one per SM sub-partition
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            kSplitWarps * ((r.n + 31) / 32) <= 4 * (int64_t)sms) {
            rk4_split_kernel<KIND><<<(unsigned)((r.n + 31) / 32), 32 * kSplitWarps, 0, s>>>(
                m, view<R>(r), make_omega<R>(omega), dt, n_steps, r2, every, ckpt, work_counters());
            return cudaGetLastError();
        }
    }
    const int block = rk4_block(rk4_kernel<R, KIND, DF>, r.n);
    const int64_t blocks = (r.n + block - 1) / block;
    rk4_kernel<R, KIND, DF><<<(unsigned)blocks, block, 0, s>>>(m, view<R>(r), make_omega<R>(omega), (R)dt,
                                                               dt, n_steps, r2, every, ckpt, work_counters());
    return cudaGetLastError();
}

template <typename R, int KIND>
static cudaError_t rk4_launch_df(const MediumParams &m, const gf_rays &r, double omega, double dt,
                                 int64_t n_steps, double radius, int64_t every, double *ckpt, cudaStream_t s)
{
    // media without blobs have nothing to evaluate in double-float
    if (m.n_blobs == 0) return rk4_launch<double, KIND, false>(m, r, omega, dt, n_steps, radius, every, ckpt, s);
    return rk4_launch<double, KIND, true>(m, r, omega, dt, n_steps, radius, every, ckpt, s);
}

template <typename R, int KIND>
static cudaError_t onshell_launch(const MediumParams &m, const gf_rays &r, const void *dir, double omega,
                                  cudaStream_t s)
{
    const int64_t blocks = (r.n + kRk4Block - 1) / kRk4Block;
    onshell_kernel<R, KIND><<<(unsigned)blocks, kRk4Block, 0, s>>>(m, view<R>(r), (const R *)dir, (R)omega);
    return cudaGetLastError();
}

#define GF_KIND_SWITCH(KIND_VAR, FN, R, ...)                                      \
    switch (KIND_VAR) {                                                            \
    case K_HOMOG: return FN<R, K_HOMOG>(__VA_ARGS__);                             \
    case K_LUNEBURG: return FN<R, K_LUNEBURG>(__VA_ARGS__);                       \
    case K_GRIN: return FN<R, K_GRIN>(__VA_ARGS__);                               \
    case K_QUADRATIC: return FN<R, K_QUADRATIC>(__VA_ARGS__);                     \
    case K_SPLINE: return FN<R, K_SPLINE>(__VA_ARGS__);                           \
    case K_COLD: return FN<R, K_COLD>(__VA_ARGS__);                               \
    default: return cudaErrorInvalidValue;                                         \
    }
#define GF_KIND_SWITCH_NO_COLD(KIND_VAR, FN, R, ...)                              \
    switch (KIND_VAR) {                                                            \
    case K_HOMOG: return FN<R, K_HOMOG>(__VA_ARGS__);                             \
    case K_LUNEBURG: return FN<R, K_LUNEBURG>(__VA_ARGS__);                       \
    case K_GRIN: return FN<R, K_GRIN>(__VA_ARGS__);                               \
    case K_QUADRATIC: return FN<R, K_QUADRATIC>(__VA_ARGS__);                     \
    case K_SPLINE: return FN<R, K_SPLINE>(__VA_ARGS__);                           \
    default: return cudaErrorInvalidValue;                                         \
    }

cudaError_t launch_rk4(const MediumParams &m, gf_precision prec, const gf_rays &r, double omega,
                       double dt, int64_t n_steps, double radius, int64_t every, double *ckpt,
                       cudaStream_t s)
{
    if (r.n == 0) return cudaSuccess;
    if (prec == GF_F64) {
        GF_KIND_SWITCH(m.kind, rk4_launch, double, m, r, omega, dt, n_steps, radius, every, ckpt, s)
    } else if (prec == GF_F64X) {
        switch (m.kind) {
        case K_HOMOG: return rk4_launch_df<double, K_HOMOG>(m, r, omega, dt, n_steps, radius, every, ckpt, s);
        case K_LUNEBURG: return rk4_launch_df<double, K_LUNEBURG>(m, r, omega, dt, n_steps, radius, every, ckpt, s);
        case K_GRIN: return rk4_launch_df<double, K_GRIN>(m, r, omega, dt, n_steps, radius, every, ckpt, s);
        case K_QUADRATIC: return rk4_launch_df<double, K_QUADRATIC>(m, r, omega, dt, n_steps, radius, every, ckpt, s);
        case K_SPLINE: return rk4_launch<double, K_SPLINE>(m, r, omega, dt, n_steps, radius, every, ckpt, s);
        case K_COLD: return rk4_launch<double, K_COLD>(m, r, omega, dt, n_steps, radius, every, ckpt, s);
        default: return cudaErrorInvalidValue;
        }
    } else {
        GF_KIND_SWITCH(m.kind, rk4_launch, float, m, r, omega, dt, n_steps, radius, every, ckpt, s)
    }
}

template <typename R, int KIND>
static cudaError_t newton_launch(const MediumParams &m, const gf_rays &r, double omega, double tol, int max_iter,
                                 cudaStream_t s)
{
    const int64_t blocks = (r.n + kRk4Block - 1) / kRk4Block;
    newton_kx_kernel<R, KIND><<<(unsigned)blocks, kRk4Block, 0, s>>>(m, view<R>(r), (R)omega, (R)tol, max_iter);
    return cudaGetLastError();
}

cudaError_t launch_newton_kx(const MediumParams &m, gf_precision prec, const gf_rays &r, double omega, double tol,
                             int max_iter, cudaStream_t s)
{
    if (r.n == 0) return cudaSuccess;
    if (prec == GF_F64 || prec == GF_F64X) {
        GF_KIND_SWITCH(m.kind, newton_launch, double, m, r, omega, tol, max_iter, s)
    } else {
        GF_KIND_SWITCH(m.kind, newton_launch, float, m, r, omega, tol, max_iter, s)
    }
}

cudaError_t launch_onshell(const MediumParams &m, gf_precision prec, const gf_rays &r, const void *dir,
                           double omega, cudaStream_t s)
{
    if (r.n == 0) return cudaSuccess;
    if (prec == GF_F64 || prec == GF_F64X) {
        GF_KIND_SWITCH_NO_COLD(m.kind, onshell_launch, double, m, r, dir, omega, s)
    } else {
        GF_KIND_SWITCH_NO_COLD(m.kind, onshell_launch, float, m, r, dir, omega, s)
    }
}

}  // namespace gf
