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
             K_QUADRATIC = GF_MED_QUADRATIC, K_SPLINE = GF_MED_SPLINE };

constexpr int kBlobStride = 5;   // device blob row: A, cx, cy, cz, s = -1 / (2 w^2)

// Medium as the kernels see it (passed by value as a kernel argument).
struct MediumParams {
    int32_t kind, n_blobs, grid_n, pad;
    double n_h2;                 // homogeneous n^2
    double n02, n02a2;           // GRIN: n0^2 and n0^2 a^2
    const double *blobs64;       // n_blobs x kBlobStride
    const float *blobs32;        // float copy of the same table
    const float4 *grid;          // grid_n^3 nodes x 2 float4
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

// ------------------------------------------------------------------ host side

void set_error(const char *fmt, ...);
gf_status cuda_status(cudaError_t e, const char *what);
gf_status check_rays(const gf_rays *r, bool need_state);
gf_status check_device_ptr(const void *p, const char *name);
const MediumParams &params_of(gf_medium m);
int device_of(gf_medium m);

// Per-translation-unit launchers (return cudaGetLastError() of the launch).
cudaError_t launch_rk4(const MediumParams &m, gf_precision prec, const gf_rays &r, double omega,
                       double dt, int64_t n_steps, double radius, int64_t every, double *ckpt,
                       cudaStream_t s);
cudaError_t launch_onshell(const MediumParams &m, gf_precision prec, const gf_rays &r,
                           const void *dir, double omega, cudaStream_t s);

// ---------------------------------------------------------------- device side

template <typename R>
__device__ __forceinline__ R dev_exp(R a);
template <>
__device__ __forceinline__ double dev_exp<double>(double a) { return exp(a); }
template <>
__device__ __forceinline__ float dev_exp<float>(float a) { return expf(a); }

template <typename R>
__device__ __forceinline__ const R *blob_table(const MediumParams &m);
template <>
__device__ __forceinline__ const double *blob_table<double>(const MediumParams &m) { return m.blobs64; }
template <>
__device__ __forceinline__ const float *blob_table<float>(const MediumParams &m) { return m.blobs32; }

// Stage the blob table into shared memory (all threads of the block call it).
template <typename R>
__device__ __forceinline__ void stage_blobs(const MediumParams &m, R *sb)
{
    const R *src = blob_table<R>(m);
    for (int j = threadIdx.x; j < m.n_blobs * kBlobStride; j += blockDim.x) sb[j] = src[j];
}

// Squared index n^2 and its gradient for an isotropic medium of kind KIND plus
// the Gaussian blobs in sb:  n^2 += A exp(s q),  grad += 2 s A exp(s q) (x - c),
// with q = |x - c|^2 and s = -1 / (2 w^2).
template <typename R, int KIND>
__device__ __forceinline__ void iso_index(const MediumParams &m, const R *__restrict__ sb, int nb,
                                          const R *x, R &n2, R *g)
{
    if constexpr (KIND == K_HOMOG) {
        n2 = (R)m.n_h2;
        g[0] = g[1] = g[2] = (R)0;
    } else if constexpr (KIND == K_LUNEBURG) {
        R r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        if (r2 <= (R)1) {
            n2 = (R)2 - r2;
            g[0] = (R)-2 * x[0];
            g[1] = (R)-2 * x[1];
            g[2] = (R)-2 * x[2];
        } else {
            n2 = (R)1;
            g[0] = g[1] = g[2] = (R)0;
        }
    } else if constexpr (KIND == K_QUADRATIC) {
        R r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        n2 = (R)2 - r2;
        g[0] = (R)-2 * x[0];
        g[1] = (R)-2 * x[1];
        g[2] = (R)-2 * x[2];
    } else {  // K_GRIN
        R c = (R)m.n02a2;
        n2 = (R)m.n02 - c * (x[1] * x[1] + x[2] * x[2]);
        g[0] = (R)0;
        g[1] = (R)-2 * c * x[1];
        g[2] = (R)-2 * c * x[2];
    }
#pragma unroll 4
    for (int j = 0; j < nb; ++j) {
        const R *b = sb + kBlobStride * j;
        R dx = x[0] - b[1], dy = x[1] - b[2], dz = x[2] - b[3];
        R q = dx * dx + dy * dy + dz * dz;
        R Ae = b[0] * dev_exp<R>(q * b[4]);
        n2 += Ae;
        R c = (R)2 * b[4] * Ae;
        g[0] += c * dx;
        g[1] += c * dy;
        g[2] += c * dz;
    }
}

// Ray right-hand side for an isotropic medium, D = |k|^2 - w^2 n^2:
//   f_x = -D_k / D_w = k / (w n^2),  f_k = D_x / D_w = w grad n^2 / (2 n^2).
// Returns false (cut-off) where n^2 <= 0; D is set either way.
template <typename R, int KIND>
__device__ __forceinline__ bool rhs_iso(const MediumParams &m, const R *__restrict__ sb, int nb,
                                        R omega, const R *y, R *f, R &D)
{
    R n2, g[3];
    iso_index<R, KIND>(m, sb, nb, y, n2, g);
    D = y[3] * y[3] + y[4] * y[4] + y[5] * y[5] - omega * omega * n2;
    if (!(n2 > (R)0)) return false;
    R inv = (R)1 / n2;
    R a = inv / omega;
    R b = (R)0.5 * omega * inv;
    f[0] = a * y[3];
    f[1] = a * y[4];
    f[2] = a * y[5];
    f[3] = b * g[0];
    f[4] = b * g[1];
    f[5] = b * g[2];
    return true;
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
                R v[7] = {(R)lo.x, (R)lo.y, (R)lo.z, (R)lo.w, (R)hi.x, (R)hi.y, (R)hi.z};
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
__device__ __forceinline__ bool rhs_spline(const MediumParams &m, R omega, const R *y, R *f, R &D)
{
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

// Dispatch on the medium kind at compile time.
template <typename R, int KIND>
struct Rhs {
    const MediumParams &m;
    const R *sb;
    int nb;
    R omega;
    __device__ __forceinline__ bool operator()(const R *y, R *f, R &D) const
    {
        if constexpr (KIND == K_SPLINE)
            return rhs_spline<R>(m, omega, y, f, D);
        else
            return rhs_iso<R, KIND>(m, sb, nb, omega, y, f, D);
    }
};

}  // namespace gf
