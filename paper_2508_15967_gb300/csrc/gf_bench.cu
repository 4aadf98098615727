// gf_bench.cu -- FMA-throughput microbenchmark behind gf_bench_fma_peak.
#include "gf_dfloat.cuh"
#include "gf_internal.cuh"
#include "../../include/gf_bench.h"

namespace gf {

template <typename R>
__global__ void __launch_bounds__(256) fma_peak_kernel(R *out, int64_t iters, R a, R b)
{
    R x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = (R)(threadIdx.x + c) * (R)1e-3;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
    }
    R s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    if (s == (R)-1) out[blockIdx.x] = s;   // never true; keeps the chains live
}

template <typename R>
static gf_status run_peak(int64_t iters, int bps, double *tflops, double *ms)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * bps;
    R *out = nullptr;
    gf_status s;
    if ((s = cuda_status(dev_alloc(&out, sizeof(R) * blocks), "cudaMalloc")) != GF_OK) return s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_peak_kernel<R><<<blocks, 256>>>(out, iters / 16 + 1, (R)0.9999999, (R)1e-7);  // warm-up
    cudaEventRecord(e0);
    fma_peak_kernel<R><<<blocks, 256>>>(out, iters, (R)0.9999999, (R)1e-7);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(out);
    if ((s = cuda_status(err == cudaSuccess ? cudaGetLastError() : err, "fma_peak_kernel")) != GF_OK)
        return s;
    *ms = t;
    *tflops = 2.0 * 8.0 * (double)iters * blocks * 256.0 / (t * 1e-3) / 1e12;
    return GF_OK;
}

__global__ void dfexp_check_kernel(const double *in, double *out, int64_t n)
{
    __shared__ float sT[2 * kDfExpN];
    stage_dfexp_table(sT);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = df_to_double(df_exp2(df_from_double(in[i]), sT));
}

__global__ void exp_check_kernel(const double *in, double *out_lib, double *out_cuda, int64_t n)
{
    __shared__ double sT[kExpTabN];
    stage_exp_table(sT);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out_lib[i] = exp2_tab_int(in[i], sT);
    out_cuda[i] = exp2(in[i]);
}

__global__ void exp_fp_check_kernel(const double *in, double *out, int64_t n)
{
    __shared__ double sT[kExpTabN];
    stage_exp_table(sT);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = exp2_tab_fp(in[i], sT);
}

__global__ void blob_gauss_check_kernel(const double *u, double *out_int, double *out_fp, int64_t n)
{
    __shared__ double sT[kExpTabN];
    stage_exp_table(sT);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double u0 = u[i], u1 = u[n + i], u2 = u[2 * n + i];
    out_int[i] = blob_gauss(u0, u1, u2, sT, false);
    out_fp[i] = blob_gauss(u0, u1, u2, sT, true);
}

__global__ void recip_check_kernel(const double *in, double *out_recip, float *out_narrow, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = in[i];
    out_recip[i] = v > 0.0 ? recip_pos(v) : 0.0;
    out_narrow[i] = narrow_trunc(v);
}

}  // namespace gf

extern "C" gf_status gf_bench_recip(const double *in, double *out_recip, float *out_narrow, int64_t n,
                                    void *stream)
{
    if (n < 0) {
        gf::set_error("gf_bench_recip: n < 0");
        return GF_ERR_INVALID_ARG;
    }
    if (n == 0) return GF_OK;
    gf_status s;
    if ((s = gf::check_device_ptr(in, "in")) != GF_OK ||
        (s = gf::check_device_ptr(out_recip, "out_recip")) != GF_OK ||
        (s = gf::check_device_ptr(out_narrow, "out_narrow")) != GF_OK)
        return s;
    gf::recip_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(in, out_recip,
                                                                                         out_narrow, n);
    return gf::cuda_status(cudaGetLastError(), "gf_bench_recip launch");
}

extern "C" gf_status gf_bench_exp(const double *in, double *out_lib, double *out_cuda, int64_t n,
                                  void *stream)
{
    if (n < 0) {
        gf::set_error("gf_bench_exp: n < 0");
        return GF_ERR_INVALID_ARG;
    }
    if (n == 0) return GF_OK;
    gf_status s;
    if ((s = gf::check_device_ptr(in, "in")) != GF_OK || (s = gf::check_device_ptr(out_lib, "out_lib")) != GF_OK ||
        (s = gf::check_device_ptr(out_cuda, "out_cuda")) != GF_OK)
        return s;
    gf::exp_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(in, out_lib, out_cuda, n);
    return gf::cuda_status(cudaGetLastError(), "gf_bench_exp launch");
}

extern "C" gf_status gf_bench_exp_fp(const double *in, double *out, int64_t n, void *stream)
{
    if (n < 0) {
        gf::set_error("gf_bench_exp_fp: n < 0");
        return GF_ERR_INVALID_ARG;
    }
    if (n == 0) return GF_OK;
    gf_status s;
    if ((s = gf::check_device_ptr(in, "in")) != GF_OK || (s = gf::check_device_ptr(out, "out")) != GF_OK) return s;
    gf::exp_fp_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(in, out, n);
    return gf::cuda_status(cudaGetLastError(), "gf_bench_exp_fp launch");
}

extern "C" gf_status gf_bench_exp_df(const double *in, double *out, int64_t n, void *stream)
{
    if (n < 0) {
        gf::set_error("gf_bench_exp_df: n < 0");
        return GF_ERR_INVALID_ARG;
    }
    if (n == 0) return GF_OK;
    gf_status s;
    if ((s = gf::check_device_ptr(in, "in")) != GF_OK || (s = gf::check_device_ptr(out, "out")) != GF_OK) return s;
    gf::dfexp_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(in, out, n);
    return gf::cuda_status(cudaGetLastError(), "gf_bench_exp_df launch");
}

extern "C" gf_status gf_bench_fma_peak(gf_precision prec, int64_t iters, int32_t blocks_per_sm,
                                       double *out_tflops, double *out_ms)
{
    if (iters <= 0 || blocks_per_sm <= 0 || out_tflops == nullptr || out_ms == nullptr) {
        gf::set_error("gf_bench_fma_peak: need iters > 0, blocks_per_sm > 0 and outputs");
        return GF_ERR_INVALID_ARG;
    }
    if (prec == GF_F64) return gf::run_peak<double>(iters, blocks_per_sm, out_tflops, out_ms);
    if (prec == GF_F32) return gf::run_peak<float>(iters, blocks_per_sm, out_tflops, out_ms);
    gf::set_error("gf_bench_fma_peak: unknown precision");
    return GF_ERR_INVALID_ARG;
}

extern "C" gf_status gf_bench_blob_gauss(const double *u, double *out_int, double *out_fp, int64_t n, void *stream)
{
    if (n < 0) {
        gf::set_error("gf_bench_blob_gauss: n < 0");
        return GF_ERR_INVALID_ARG;
    }
    if (n == 0) return GF_OK;
    gf_status s;
    if ((s = gf::check_device_ptr(u, "u")) != GF_OK || (s = gf::check_device_ptr(out_int, "out_int")) != GF_OK ||
        (s = gf::check_device_ptr(out_fp, "out_fp")) != GF_OK)
        return s;
    gf::blob_gauss_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(u, out_int, out_fp,
                                                                                              n);
    return gf::cuda_status(cudaGetLastError(), "gf_bench_blob_gauss launch");
}
