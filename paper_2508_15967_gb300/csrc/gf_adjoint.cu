// gf_adjoint.cu -- discrete adjoint of the fixed-step RK4 ray trace with
// respect to the blob amplitudes theta_j = A_j of an isotropic medium.
//
// For one RK4 step with stage points Y_1 = y, Y_i = y + a_i dt K_{i-1},
// K_i = f(Y_i), y' = y + dt sum_i b_i K_i (a = 0, 1/2, 1/2, 1; b = 1/6, 1/3,
// 1/3, 1/6) and lambda = dL/dy', the reverse sweep is, for i = 4 .. 1,
//     Kbar_i = dt b_i lambda + dt a_{i+1} Ybar_{i+1}      (no second term at i = 4)
//     Ybar_i = J_f(Y_i)^T Kbar_i,    thetabar += (df/dtheta)(Y_i)^T Kbar_i
// and then lambda <- lambda + sum_i Ybar_i.
//
// For f = (a k, b grad n^2) with a = 1/(w n^2), b = w/(2 n^2), u = 1/n^2 and
// g = grad n^2, H = Hess n^2, G_j = exp(s_j |x - c_j|^2), s_j = -1/(2 w_j^2):
//     xbar = b H Kbar_k + C g,   kbar = a Kbar_x,
//     C = -u (a k.Kbar_x + b g.Kbar_k),
//     thetabar_j += G_j (C + 2 b s_j (x - c_j).Kbar_k),
//     H Kbar_k = H_base Kbar_k + sum_j A_j G_j 2 s_j (2 s_j ((x - c_j).Kbar_k)(x - c_j) + Kbar_k).
//
// Checkpoints of the forward trace every E steps bound the memory.  Each
// segment is recomputed forward from its checkpoint with the forward kernel's
// own arithmetic (the same evaluator and the same explicitly rounded RK4
// combination, so the recomputed states are the forward trace's bits: each
// segment ends exactly on the next checkpoint, which the work counters
// check), storing only every stage's point, n^2 and grad n^2.  The reverse
// sweep then evaluates the Gaussians again, and with them the blob terms of
// the vector-Jacobian product, in double-float arithmetic (float pairs,
// ~48-bit significands) on the FP32 pipes, which the FP64-bound
// recomputation leaves idle: the FP64 pipe carries only the per-stage
// algebra.  The products enter the gradient and lambda as derivative factors
// with ~1e-14 relative error, far inside the 1e-9 gradient gate; the
// trajectory itself is the FP64 recomputation.  thetabar_j of every ray is
// accumulated in a per-ray global array (L2-resident) with fire-and-forget
// atomic adds -- one thread per address, so the adds apply in program order
// and the sums are deterministic -- and reduced over rays in a fixed order.
#include <cmath>

#include "gf_dfloat.cuh"

namespace gf {

constexpr int kAdjBlock = 64;
constexpr int kStageVals = 10;   // Y (6), n^2, grad n^2 (3)
constexpr int kSwRow = 12;       // sweep row: c (hi 3, lo 3), then the pairs of s/ln2, 2 s and 2 s A

struct AdjScratch {
    double *tb;         // nb x n: thetabar_j of every ray, reduced over rays at the end
    double *stage;      // every x 4 x kStageVals x n
};

// H_base v for the base index law (Luneburg inside / quadratic: -2 I; GRIN:
// diag(0, -2c, -2c); homogeneous and Luneburg outside: 0).
template <int KIND>
__device__ __forceinline__ void base_hess_vec(const MediumParams &m, const double *x, const double *v,
                                              double *out)
{
    if constexpr (KIND == K_LUNEBURG) {
        const double h = norm2_fixed(x) <= 1.0 ? -2.0 : 0.0;
        out[0] = h * v[0];
        out[1] = h * v[1];
        out[2] = h * v[2];
    } else if constexpr (KIND == K_QUADRATIC) {
        out[0] = -2.0 * v[0];
        out[1] = -2.0 * v[1];
        out[2] = -2.0 * v[2];
    } else if constexpr (KIND == K_GRIN) {
        out[0] = 0.0;
        out[1] = -2.0 * m.n02a2 * v[1];
        out[2] = -2.0 * m.n02a2 * v[2];
    } else {
        out[0] = out[1] = out[2] = 0.0;
    }
}

// Sweep rows in shared memory: the medium's double-float rows (c, s/ln2,
// 2 s A) with the A pair replaced by 2 s, split from the plain FP64 rows.
__device__ __forceinline__ void stage_sweep_rows(const MediumParams &m, float *sw)
{
    for (int j = threadIdx.x; j < m.n_blobs; j += blockDim.x) {
        const float *src = m.dfrows + kDfBlobStride * j;
        float *dst = sw + kSwRow * j;
        for (int f = 0; f < kSwRow; ++f) dst[f] = src[f];
        const dfl t = df_from_double(m.blobs64[kBlobStride * j + 5]);   // 2 s
        dst[8] = t.hi;
        dst[9] = t.lo;
    }
}

// Warp-aggregated add of per-thread counts to counters[0..3].
__device__ __forceinline__ void add_adjoint_work(unsigned long long *counters, const long long *v)
{
    if (counters == nullptr) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        long long x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x != 0) atomicAdd(counters + k, (unsigned long long)x);
    }
}

template <int KIND>
// 8 resident blocks of 64 per SM (registers capped at 128, 24 KB of tables per
// block): the 65,536-ray adjoint workload (1,024 blocks) is resident in one
// wave on 152 SMs, at most 7 blocks against 6.74 on average per SM (blocks of
// 128 would put 4 against 3.37: 84% of the SMs' time used instead of 96%).
__global__ void __launch_bounds__(kAdjBlock, 8) adjoint_kernel(
    const MediumParams m, const int64_t n, const Omega<double> om, const double dt, const int64_t n_steps,
    const int64_t every, const double *__restrict__ ckpt, const int32_t *__restrict__ steps_done,
    const double *__restrict__ lambda, const int64_t ld, double *__restrict__ dy0, const AdjScratch S,
    unsigned long long *counters)
{
    __shared__ double sbs[kBlobStride * GF_MAX_BLOBS];   // scaled FP64 rows (recomputation)
    __shared__ double sT[kExpTabN];                      // 2^(j/2048) (both passes)
    __shared__ float sp[4 * GF_MAX_BLOBS];               // FP32 pre-test rows (recomputation)
    __shared__ float sw[kSwRow * GF_MAX_BLOBS];          // double-float sweep rows
    const int nb = m.n_blobs;
    stage_blobs<double>(m, sbs);
    stage_pretest(m, sp);
    stage_exp_table(sT);
    stage_sweep_rows(m, sw);
    __syncthreads();
    const DfTabFromDouble dT{sT};   // the sweep's table entries as float pairs
    EvalCtx<double> cx;
    cx.T = sT;
    cx.pre = sp;
    cx.exp_fp = true;   // the sweep keeps the FP32 pipes busy: the FP64-pipe form (same bits)
    long long work[4] = {0, 0, 0, 0};   // recomputed evaluations, their blob terms, swept blob terms,
                                        // segment ends that differ from the next checkpoint
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        double *acc_t = S.tb + i;   // thetabar_j of this ray at acc_t[j * n] (zeroed before the launch)
        const int sd = steps_done[i];
        double lam[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) lam[c] = lambda[c * ld + i];
        const double h2 = dt * 0.5, h6 = dt / 6.0, h3 = dt / 3.0;
        const int64_t nseg = (n_steps + every - 1) / every;
        for (int64_t seg = nseg - 1; seg >= 0; --seg) {
            const int64_t s0 = seg * every;
            if (s0 >= sd) continue;
            const int ns = (int)min(every, (int64_t)sd - s0);
            double y[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) y[c] = ckpt[(seg * 6 + c) * n + i];
            // ---- forward recomputation of the segment (the forward kernel's step), storing every stage
            for (int s = 0; s < ns; ++s) {
                double K[6], acc[6], Y[6], D;
                double *Ss = S.stage + ((int64_t)(s * 4) * kStageVals) * n + i;
#pragma unroll
                for (int c = 0; c < 6; ++c) Y[c] = y[c];
                // a rolled stage loop: one copy of the evaluator in the code
#pragma unroll 1
                for (int st = 0; st < 4; ++st) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) Ss[c * n] = Y[c];
                    double ng[4];
                    rhs_iso<double, KIND, false>(m, sbs, nb, om, Y, K, D, cx, 1, ng);
#pragma unroll
                    for (int c = 0; c < 4; ++c) Ss[(6 + c) * n] = ng[c];
                    Ss += (int64_t)kStageVals * n;
                    if (st < 3) {
                        const double hj = st == 2 ? dt : h2;
#pragma unroll
                        for (int c = 0; c < 6; ++c) {
                            acc[c] = st == 0 ? K[c] : rk_acc2(acc[c], K[c]);
                            Y[c] = rk_axpy(hj, K[c], y[c]);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < 6; ++c) y[c] = __dadd_rn(y[c], rk_inc(h6, acc[c], K[c]));
                    }
                }
            }
            work[0] += 4 * (long long)ns;
            if ((seg + 1) * every < sd) {   // the forward trace wrote the next checkpoint: same bits
#pragma unroll
                for (int c = 0; c < 6; ++c)
                    work[3] += __double_as_longlong(y[c]) != __double_as_longlong(ckpt[((seg + 1) * 6 + c) * n + i]);
            }
            // ---- reverse sweep over the segment
            for (int s = ns - 1; s >= 0; --s) {
                double ybar_next[6] = {0, 0, 0, 0, 0, 0}, ysum[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 1
                for (int st = 3; st >= 0; --st) {
                    // Kbar_i = dt b_i lambda + dt a_{i+1} Ybar_{i+1}
                    const double b_i = (st == 0 || st == 3) ? h6 : h3, a_next = st == 2 ? dt : h2;
                    double Kb[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) Kb[c] = st < 3 ? fma(a_next, ybar_next[c], b_i * lam[c]) : b_i * lam[c];
                    const double *Ss = S.stage + ((int64_t)(s * 4 + st) * kStageVals) * n + i;
                    double Y[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) Y[c] = Ss[c * n];
                    const double n2 = Ss[6 * n], g0 = Ss[7 * n], g1 = Ss[8 * n], g2 = Ss[9 * n];
                    const double u = recip_pos(n2);
                    const double a = u * om.inv_w, bq = om.half_w * u;
                    const double C = -u * (a * (Y[3] * Kb[0] + Y[4] * Kb[1] + Y[5] * Kb[2]) +
                                           bq * (g0 * Kb[3] + g1 * Kb[4] + g2 * Kb[5]));
                    double HK[3];
                    base_hess_vec<KIND>(m, Y, Kb + 3, HK);
                    // blob terms in double-float
                    const dfl X0 = df_from_double(Y[0]), X1 = df_from_double(Y[1]), X2 = df_from_double(Y[2]);
                    const dfl B0 = df_from_double(Kb[3]), B1 = df_from_double(Kb[4]), B2 = df_from_double(Kb[5]);
                    const dfl Cd = df_from_double(C), Bq = df_from_double(bq);
                    dfl H0 = {0.f, 0.f}, H1 = {0.f, 0.f}, H2 = {0.f, 0.f};
                    for (int j = 0; j < nb; ++j) {
                        const float *w = sw + kSwRow * j;
                        const float ex = X0.hi - w[0], ey = X1.hi - w[1], ez = X2.hi - w[2];
                        if ((ex * ex + ey * ey + ez * ez) * w[6] < -kDfPreCull2) continue;
                        const dfl d0 = df_add(X0, dfl{-w[0], -w[3]});
                        const dfl d1 = df_add(X1, dfl{-w[1], -w[4]});
                        const dfl d2 = df_add(X2, dfl{-w[2], -w[5]});
                        const dfl q = df_add_sloppy(df_add_sloppy(df_sqr(d0), df_sqr(d1)), df_sqr(d2));
                        const dfl ea = df_mul(dfl{w[6], w[7]}, q);
                        if (ea.hi < (float)kBlobCull2) continue;
                        const dfl E = df_exp2_tab(ea, dT);                                // G_j
                        const dfl dK = df_add(df_add(df_mul(d0, B0), df_mul(d1, B1)), df_mul(d2, B2));
                        const dfl wv = df_mul(dfl{w[8], w[9]}, dK);                        // 2 s (x - c).Kbar_k
                        const dfl v = df_mul(E, df_add(Cd, df_mul(Bq, wv)));
                        atomicAdd(acc_t + (int64_t)j * n, df_to_double(v));
                        const dfl BE = df_mul(dfl{w[10], w[11]}, E);                       // 2 s A G
                        H0 = df_add_sloppy(H0, df_mul(BE, df_add(df_mul(wv, d0), B0)));
                        H1 = df_add_sloppy(H1, df_mul(BE, df_add(df_mul(wv, d1), B1)));
                        H2 = df_add_sloppy(H2, df_mul(BE, df_add(df_mul(wv, d2), B2)));
                        ++work[2];
                    }
                    HK[0] += df_to_double(H0);
                    HK[1] += df_to_double(H1);
                    HK[2] += df_to_double(H2);
                    double yb[6];
                    yb[0] = bq * HK[0] + C * g0;
                    yb[1] = bq * HK[1] + C * g1;
                    yb[2] = bq * HK[2] + C * g2;
                    yb[3] = a * Kb[0];
                    yb[4] = a * Kb[1];
                    yb[5] = a * Kb[2];
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        ysum[c] += yb[c];
                        ybar_next[c] = yb[c];
                    }
                }
#pragma unroll
                for (int c = 0; c < 6; ++c) lam[c] += ysum[c];
            }
        }
        if (dy0 != nullptr) {
#pragma unroll
            for (int c = 0; c < 6; ++c) dy0[c * ld + i] = lam[c];
        }
    }
    work[1] = cx.live;
    add_adjoint_work(counters, work);
}

// dL/dtheta_j = sum over rays of thetabar_j, one block per blob in a fixed
// order (each thread a strided partial sum, then a tree): deterministic.
constexpr int kRedBlock = 256;

__global__ void __launch_bounds__(kRedBlock) adjoint_reduce_kernel(const double *__restrict__ tb, int64_t n,
                                                                   double *__restrict__ out)
{
    __shared__ double part[kRedBlock];
    const int j = blockIdx.x;
    double sum = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kRedBlock) sum += tb[(int64_t)j * n + i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int w = kRedBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = part[0];
}

size_t adjoint_scratch_bytes(int nb, int64_t n, int64_t every)
{
    return sizeof(double) * ((size_t)nb * n + (size_t)every * 4 * kStageVals * (size_t)n) + 256;
}

cudaError_t launch_adjoint(const MediumParams &m, int64_t n, double omega, double dt, int64_t n_steps,
                           int64_t every, const double *ckpt, const int32_t *steps_done, const double *lambda,
                           int64_t ld, double *dtheta, double *dy0, void *scratch, cudaStream_t s)
{
    const int nb = m.n_blobs;
    const int64_t blocks = (n + kAdjBlock - 1) / kAdjBlock;
    char *base = (char *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
    AdjScratch S;
    S.tb = (double *)base;
    S.stage = S.tb + (int64_t)nb * n;
    cudaError_t e = cudaMemsetAsync(S.tb, 0, sizeof(double) * (size_t)nb * n, s);
    if (e != cudaSuccess) return e;
    const Omega<double> om = make_omega<double>(omega);
    unsigned long long *counters = work_counters();
#define GF_ADJ(K)                                                                                          \
    case K:                                                                                                \
        adjoint_kernel<K><<<(unsigned)blocks, kAdjBlock, 0, s>>>(m, n, om, dt, n_steps, every, ckpt,        \
                                                                 steps_done, lambda, ld, dy0, S, counters); \
        break;
    switch (m.kind) {
        GF_ADJ(K_HOMOG)
        GF_ADJ(K_LUNEBURG)
        GF_ADJ(K_GRIN)
        GF_ADJ(K_QUADRATIC)
    default:
        return cudaErrorInvalidValue;
    }
#undef GF_ADJ
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nb > 0) adjoint_reduce_kernel<<<nb, kRedBlock, 0, s>>>(S.tb, n, dtheta);
    return cudaGetLastError();
}

}  // namespace gf

// ------------------------------------------------ allocation-free entry point

namespace gf {

// Fixed scratch of gf_trace_adjoint_static.  It is part of this file's device
// module, so every GPU on which the module is loaded holds it until the
// process exits.
constexpr size_t kStaticAdjointScratchBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_adjoint_scratch[kStaticAdjointScratchBytes];

// Device address of g_adjoint_scratch in the current device's context, looked
// up on every call (host code cannot use the symbol itself as a device
// address).  Not cached: a context that is torn down and created again (for
// example after cudaDeviceReset) loads the module anew, and the array may
// then sit at another address.  The first lookup on a device may load this
// file's module (lazy loading), which maps the array.
static gf_status static_scratch(void **out)
{
    void *p = nullptr;
    gf_status s = cuda_status(cudaGetSymbolAddress(&p, g_adjoint_scratch), "cudaGetSymbolAddress");
    if (s != GF_OK) return s;
    *out = p;
    return GF_OK;
}

}  // namespace gf

extern "C" gf_status gf_trace_adjoint_static(gf_medium m, int64_t n, double omega, double dt,
                                             int64_t n_steps, int64_t checkpoint_every,
                                             const double *ckpt, const int32_t *steps_done,
                                             const double *lambda, int64_t ld, double *dL_dtheta,
                                             double *dL_dy0, void *stream)
{
    using namespace gf;
    gf_status s;
    if (m == nullptr) {
        set_error("gf_trace_adjoint_static: medium is NULL");
        return GF_ERR_INVALID_ARG;
    }
    int dev = -1;
    if ((s = cuda_status(cudaGetDevice(&dev), "cudaGetDevice")) != GF_OK) return s;
    if (dev != device_of(m)) {
        set_error("gf_trace_adjoint_static: medium lives on device %d, current device is %d", device_of(m), dev);
        return GF_ERR_INVALID_ARG;
    }
    const MediumParams &p = params_of(m);
    if (p.kind == K_SPLINE || p.kind == K_COLD || p.n_blobs < 1) {
        set_error("gf_trace_adjoint_static: needs an isotropic medium with at least one blob");
        return GF_ERR_INVALID_ARG;
    }
    if (n < 0 || ld < n || n_steps < 0 || checkpoint_every < 1 || checkpoint_every > 4096 ||
        !(omega > 0) || !std::isfinite(omega) || !(dt > 0) || !std::isfinite(dt)) {
        set_error("gf_trace_adjoint_static: need n >= 0, ld >= n, n_steps >= 0, "
                  "1 <= checkpoint_every <= 4096, omega > 0, dt > 0");
        return GF_ERR_INVALID_ARG;
    }
    const size_t need = adjoint_scratch_bytes(p.n_blobs, n, checkpoint_every);
    if (need > kStaticAdjointScratchBytes) {
        set_error("gf_trace_adjoint_static: %lld rays with %d blobs and checkpoints every %lld steps need "
                  "%zu bytes of scratch; the fixed array holds %zu (use fewer rays per call, a shorter "
                  "checkpoint interval, or gf_trace_adjoint)",
                  (long long)n, p.n_blobs, (long long)checkpoint_every, need, kStaticAdjointScratchBytes);
        return GF_ERR_INVALID_ARG;
    }
    if ((s = check_device_ptr(dL_dtheta, "dL_dtheta")) != GF_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // the lookup comes first, so that a call with n = 0 serves as the warm-up
    // call that loads the module on this device
    void *scratch = nullptr;
    if ((s = static_scratch(&scratch)) != GF_OK) return s;
    if (n == 0)
        return cuda_status(cudaMemsetAsync(dL_dtheta, 0, sizeof(double) * p.n_blobs, st),
                           "gf_trace_adjoint_static memset");
    if ((s = check_device_ptr(ckpt, "ckpt")) != GF_OK || (s = check_device_ptr(steps_done, "steps_done")) != GF_OK ||
        (s = check_device_ptr(lambda, "lambda")) != GF_OK)
        return s;
    if (dL_dy0 && (s = check_device_ptr(dL_dy0, "dL_dy0")) != GF_OK) return s;
    // every scratch word the kernels read is written earlier in the same call
    // (block partials, then the stage values of each segment), so nothing
    // needs clearing between calls
    return cuda_status(launch_adjoint(p, n, omega, dt, n_steps, checkpoint_every, ckpt, steps_done, lambda, ld,
                                      dL_dtheta, dL_dy0, scratch, st),
                       "gf_trace_adjoint_static launch");
}
