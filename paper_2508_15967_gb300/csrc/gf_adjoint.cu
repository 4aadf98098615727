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
// Checkpoints of the forward trace every E steps bound the memory: each
// segment is recomputed forward from its checkpoint, storing for every step
// and stage Y_i, n^2, g and all G_j in scratch, then swept in reverse without
// re-evaluating any exponential.  Per-thread thetabar columns live in shared
// memory and are reduced block -> grid in a fixed order (deterministic).
#include <cmath>
#include <mutex>

#include "gf_internal.cuh"

namespace gf {

constexpr int kAdjBlock = 64;
constexpr int kStageVals = 10;   // Y (6), n^2, g (3)

struct AdjScratch {
    double *tb;         // nb x n: thetabar_j of every ray, reduced over rays at the end
    double *stage;      // every x 4 x kStageVals x n
    double *G;          // every x 4 x nb x n
};

template <int KIND>
__device__ __forceinline__ void base_index(const MediumParams &m, const double *x, double &n2, double *g)
{
    EvalCtx<double> cx;
    iso_index<double, KIND>(m, nullptr, 0, x, n2, g, cx);
}

// H_base v for the base index law (Luneburg inside / quadratic: -2 I; GRIN:
// diag(0, -2c, -2c); homogeneous and Luneburg outside: 0).
template <int KIND>
__device__ __forceinline__ void base_hess_vec(const MediumParams &m, const double *x, const double *v,
                                              double *out)
{
    if constexpr (KIND == K_LUNEBURG) {
        const double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        const double h = r2 <= 1.0 ? -2.0 : 0.0;
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

template <int KIND>
// 7 resident blocks of 64 per SM (registers capped at 146): the 65,536-ray
// adjoint workload (2,048 warps) is resident in one wave on 152 SMs.
__global__ void __launch_bounds__(kAdjBlock, 7) adjoint_kernel(
    const MediumParams m, const int64_t n, const double omega, const double dt, const int64_t n_steps,
    const int64_t every, const double *__restrict__ ckpt, const int32_t *__restrict__ steps_done,
    const double *__restrict__ lambda, const int64_t ld, double *__restrict__ dy0, const AdjScratch S)
{
    __shared__ double sb[kBlobStride * GF_MAX_BLOBS];    // plain rows (reverse sweep)
    __shared__ double sbs[kBlobStride * GF_MAX_BLOBS];   // scaled rows (recompute)
    __shared__ double sT[kExpTabN];
    __shared__ float sp[4 * GF_MAX_BLOBS];               // FP32 pre-test rows (recompute)
    const int nb = m.n_blobs;
    for (int j = threadIdx.x; j < nb * kBlobStride; j += blockDim.x) {
        sb[j] = m.blobs64[j];
        sbs[j] = m.blobs64s[j];
    }
    for (int j = threadIdx.x; j < nb * 4; j += blockDim.x) sp[j] = m.pre32[j];
    stage_exp_table(sT);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        double *acc_t = S.tb + i;   // thetabar_j of this ray at acc_t[j * n]
        for (int j = 0; j < nb; ++j) acc_t[(int64_t)j * n] = 0.0;
        const int sd = steps_done[i];
        double lam[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) lam[c] = lambda[c * ld + i];
        const double aa[4] = {0.0, 0.5 * dt, 0.5 * dt, dt};
        const double bb[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};
        const int64_t nseg = (n_steps + every - 1) / every;
        for (int64_t seg = nseg - 1; seg >= 0; --seg) {
            const int64_t s0 = seg * every;
            if (s0 >= sd) continue;
            const int ns = (int)min(every, (int64_t)sd - s0);
            double y[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) y[c] = ckpt[(seg * 6 + c) * n + i];
            // ---- forward recompute of the segment, storing every stage
            for (int s = 0; s < ns; ++s) {
                double K[6], acc[6];
#pragma unroll
                for (int st = 0; st < 4; ++st) {
                    double Y[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) Y[c] = st == 0 ? y[c] : y[c] + aa[st] * K[c];
                    double n2, g[3];
                    base_index<KIND>(m, Y, n2, g);
                    // blob terms with the forward evaluator's arithmetic (scaled rows,
                    // FP32 pre-test); negligible terms (see kBlobCull2) are stored as G = 0
                    double *Gs = S.G + ((int64_t)(s * 4 + st) * nb) * n + i;
                    const PreX px = pretest_point(m, Y);
                    int live = 0;
                    for (int j = 0; j < nb; ++j)
                        Gs[(int64_t)j * n] = (px.on && pretest_negligible(sp + 4 * j, 1, px))
                                                 ? 0.0
                                                 : blob_term_scaled(sbs + kBlobStride * j, 1, Y, n2, g, sT, live);
                    double *Ss = S.stage + ((int64_t)(s * 4 + st) * kStageVals) * n + i;
#pragma unroll
                    for (int c = 0; c < 6; ++c) Ss[c * n] = Y[c];
                    Ss[6 * n] = n2;
                    Ss[7 * n] = g[0];
                    Ss[8 * n] = g[1];
                    Ss[9 * n] = g[2];
                    const double inv = recip_pos(n2);
                    const double a = inv / omega, bq = 0.5 * omega * inv;
                    K[0] = a * Y[3];
                    K[1] = a * Y[4];
                    K[2] = a * Y[5];
                    K[3] = bq * g[0];
                    K[4] = bq * g[1];
                    K[5] = bq * g[2];
#pragma unroll
                    for (int c = 0; c < 6; ++c) acc[c] = st == 0 ? K[c] : (st == 3 ? acc[c] + K[c] : acc[c] + 2.0 * K[c]);
                }
#pragma unroll
                for (int c = 0; c < 6; ++c) y[c] = y[c] + (dt / 6.0) * acc[c];
            }
            // ---- reverse sweep over the segment
            for (int s = ns - 1; s >= 0; --s) {
                double ybar_next[6] = {0, 0, 0, 0, 0, 0}, ysum[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
                for (int st = 3; st >= 0; --st) {
                    double Kb[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) Kb[c] = bb[st] * lam[c] + (st < 3 ? aa[st + 1] * ybar_next[c] : 0.0);
                    const double *Ss = S.stage + ((int64_t)(s * 4 + st) * kStageVals) * n + i;
                    double Y[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) Y[c] = Ss[c * n];
                    const double n2 = Ss[6 * n], g0 = Ss[7 * n], g1 = Ss[8 * n], g2 = Ss[9 * n];
                    const double u = recip_pos(n2);
                    const double a = u / omega, bq = 0.5 * omega * u;
                    const double C = -u * (a * (Y[3] * Kb[0] + Y[4] * Kb[1] + Y[5] * Kb[2]) +
                                           bq * (g0 * Kb[3] + g1 * Kb[4] + g2 * Kb[5]));
                    double HK[3];
                    base_hess_vec<KIND>(m, Y, Kb + 3, HK);
                    const double *Gs = S.G + ((int64_t)(s * 4 + st) * nb) * n + i;
                    for (int j = 0; j < nb; ++j) {
                        const double G = Gs[(int64_t)j * n];
                        // negligible term (stored as +0): no contribution; tested on the
                        // bit pattern, since an FP64 compare would occupy the FP64 pipe
                        if (__double_as_longlong(G) == 0ll) continue;
                        const double *b = sb + kBlobStride * j;
                        const double dx = Y[0] - b[1], dy = Y[1] - b[2], dz = Y[2] - b[3];
                        const double dK = dx * Kb[3] + dy * Kb[4] + dz * Kb[5];
                        const double s2 = b[5];
                        acc_t[(int64_t)j * n] += G * (C + bq * s2 * dK);
                        const double t = s2 * b[0] * G;
                        const double w = s2 * dK;
                        HK[0] += t * (w * dx + Kb[3]);
                        HK[1] += t * (w * dy + Kb[4]);
                        HK[2] += t * (w * dz + Kb[5]);
                    }
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
    return sizeof(double) * ((size_t)nb * n + (size_t)every * 4 * (kStageVals + nb) * (size_t)n) + 256;
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
    S.G = S.stage + every * 4 * kStageVals * n;
#define GF_ADJ(K)                                                                                      \
    case K:                                                                                            \
        adjoint_kernel<K><<<(unsigned)blocks, kAdjBlock, 0, s>>>(m, n, omega, dt, n_steps, every, ckpt, \
                                                                 steps_done, lambda, ld, dy0, S);     \
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
    cudaError_t e = cudaGetLastError();
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

constexpr int kMaxStaticDevices = 64;
static std::mutex g_static_mutex;
static void *g_static_ptr[kMaxStaticDevices] = {};

// Device address of g_adjoint_scratch on the current device, looked up once
// per device (host code cannot use the symbol itself as a device address).
static gf_status static_scratch(void **out)
{
    int dev = -1;
    gf_status s = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != GF_OK) return s;
    if (dev < 0 || dev >= kMaxStaticDevices) {
        set_error("gf_trace_adjoint_static: device ordinal %d >= %d", dev, kMaxStaticDevices);
        return GF_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (g_static_ptr[dev] == nullptr) {
        void *p = nullptr;
        if ((s = cuda_status(cudaGetSymbolAddress(&p, g_adjoint_scratch), "cudaGetSymbolAddress")) != GF_OK)
            return s;
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
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
    if (n == 0)
        return cuda_status(cudaMemsetAsync(dL_dtheta, 0, sizeof(double) * p.n_blobs, st),
                           "gf_trace_adjoint_static memset");
    if ((s = check_device_ptr(ckpt, "ckpt")) != GF_OK || (s = check_device_ptr(steps_done, "steps_done")) != GF_OK ||
        (s = check_device_ptr(lambda, "lambda")) != GF_OK)
        return s;
    if (dL_dy0 && (s = check_device_ptr(dL_dy0, "dL_dy0")) != GF_OK) return s;
    void *scratch = nullptr;
    if ((s = static_scratch(&scratch)) != GF_OK) return s;
    // every scratch word the kernels read is written earlier in the same call
    // (block partials, then the stage values of each segment), so nothing
    // needs clearing between calls
    return cuda_status(launch_adjoint(p, n, omega, dt, n_steps, checkpoint_every, ckpt, steps_done, lambda, ld,
                                      dL_dtheta, dL_dy0, scratch, st),
                       "gf_trace_adjoint_static launch");
}
