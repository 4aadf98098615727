// gf_api.cu -- host side of the C ABI declared in include/gf.h: error
// reporting, argument validation, medium objects and the RK4 / on-shell
// entry points.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "gf_internal.cuh"

namespace gf {

static thread_local std::string g_err;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

// Fault injection (gf_fault_inject): the number of further successful checked
// CUDA calls after which one reports a failure; 0 = disarmed.
static std::atomic<long long> g_inject{0};

gf_status cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) {
        long long n = g_inject.load();
        while (n > 0 && !g_inject.compare_exchange_weak(n, n - 1)) {
        }
        if (n == 1) {
            set_error("%s: injected fault (gf_fault_inject)", what);
            return GF_ERR_CUDA;
        }
        return GF_OK;
    }
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    if (e == cudaErrorMemoryAllocation) return GF_ERR_OOM;
    return GF_ERR_CUDA;
}

// Device allocations of the library, with their sizes: every allocation the
// library makes goes through dev_alloc / dev_free, so that tests can check
// that error paths release what they took (gf_bench_live_allocations).
static std::mutex g_alloc_mutex;
static std::unordered_map<void *, size_t> g_allocs;
static size_t g_alloc_bytes = 0;

cudaError_t dev_alloc(void **p, size_t bytes)
{
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        g_allocs[*p] = bytes;
        g_alloc_bytes += bytes;
    }
    return e;
}

void dev_free(void *p)
{
    if (p == nullptr) return;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        auto it = g_allocs.find(p);
        if (it != g_allocs.end()) {
            g_alloc_bytes -= it->second;
            g_allocs.erase(it);
        }
    }
    cudaFree(p);
}

// A pointer the kernels may dereference: device or managed memory, on any
// device visible to the current context.  Host and unregistered pointers
// are rejected before any launch.
gf_status check_device_ptr(const void *p, const char *name)
{
    if (p == nullptr) {
        set_error("%s is NULL", name);
        return GF_ERR_INVALID_ARG;
    }
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("%s: cudaPointerGetAttributes failed: %s", name, cudaGetErrorString(e));
        return GF_ERR_INVALID_ARG;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
        set_error("%s is not device memory", name);
        return GF_ERR_INVALID_ARG;
    }
    return GF_OK;
}

gf_status check_rays(const gf_rays *r, bool need_state)
{
    if (r == nullptr) {
        set_error("rays is NULL");
        return GF_ERR_INVALID_ARG;
    }
    if (r->n < 0 || r->ld < r->n || r->n > (int64_t)INT32_MAX * 64) {
        set_error("rays: need 0 <= n <= ld (n=%lld, ld=%lld)", (long long)r->n, (long long)r->ld);
        return GF_ERR_INVALID_ARG;
    }
    if (r->n == 0) return GF_OK;
    gf_status s;
    if ((s = check_device_ptr(r->y, "rays.y")) != GF_OK) return s;
    if ((s = check_device_ptr(r->status, "rays.status")) != GF_OK) return s;
    if (need_state) {
        if ((s = check_device_ptr(r->t, "rays.t")) != GF_OK) return s;
        if ((s = check_device_ptr(r->steps, "rays.steps")) != GF_OK) return s;
        if (r->d_res && (s = check_device_ptr(r->d_res, "rays.d_res")) != GF_OK) return s;
        if (r->d_max && (s = check_device_ptr(r->d_max, "rays.d_max")) != GF_OK) return s;
    }
    return GF_OK;
}

static unsigned long long *g_work_counters = nullptr;
unsigned long long *work_counters() { return g_work_counters; }

const MediumParams &params_of(gf_medium m) { return m->p; }
// scaled FP64 rows (what the FP64 evaluator reads)
const double *medium_device_blobs(gf_medium m) { return m->p.blobs64s; }
int device_of(gf_medium m) { return m->device; }

static gf_status check_medium(gf_medium m)
{
    if (m == nullptr) {
        set_error("medium is NULL");
        return GF_ERR_INVALID_ARG;
    }
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != m->device) {
        set_error("medium lives on device %d, current device is %d", m->device, dev);
        return GF_ERR_INVALID_ARG;
    }
    return GF_OK;
}

static void free_medium(gf_medium m)
{
    dev_free(m->d_blobs64);
    dev_free(m->d_blobs32);
    dev_free(m->d_grid);
    if (m->jit_lib) cudaLibraryUnload(m->jit_lib);
    delete m;
}

// A_j in the plain rows, A_j and -2 ln2 sigma_j A_j in the scaled rows
// (double and float), and the (hi, lo) pairs of A_j and 2 s_j A_j in the
// double-float rows.
__global__ void set_amplitudes_kernel(double *b64, float *b32, const double *A, int nb)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nb) {
        double a = A[j];
        b64[kBlobStride * j] = a;
        double *sc = b64 + kBlobStride * (nb + j);
        sc[4] = a;
        sc[5] = (kNeg2Ln2 * sc[0]) * a;
        b32[kBlobStride * j + 4] = (float)sc[4];
        b32[kBlobStride * j + 5] = (float)sc[5];
        float *dfr = b32 + (kBlobStride + 4) * nb + kDfRowFloats * j;   // A and 2 s A pairs
        const double two_sa = (2.0 * b64[kBlobStride * j + 4]) * a;
        const float hi = __double2float_rn(a);
        dfr[8] = hi;
        dfr[9] = __double2float_rn(a - (double)hi);
        const float hi2 = __double2float_rn(two_sa);
        dfr[10] = hi2;
        dfr[11] = __double2float_rn(two_sa - (double)hi2);
    }
}

}  // namespace gf

using namespace gf;

extern "C" {

const char *gf_last_error(void) { return g_err.c_str(); }

int32_t gf_version(void) { return 100; }

gf_status gf_fault_inject(int64_t n)
{
    g_inject.store(n > 0 ? (long long)n : 0);
    return GF_OK;
}

int64_t gf_bench_live_allocations(size_t *bytes)
{
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    if (bytes != nullptr) *bytes = g_alloc_bytes;
    return (int64_t)g_allocs.size();
}

gf_status gf_medium_create(const gf_medium_desc *d, gf_medium *out)
{
    if (d == nullptr || out == nullptr) {
        set_error("gf_medium_create: desc and out must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (d->kind < GF_MED_HOMOG || d->kind > GF_MED_COLD || d->reserved != 0 || d->reserved2 != 0) {
        set_error("gf_medium_create: unknown kind %d or reserved != 0", d->kind);
        return GF_ERR_INVALID_ARG;
    }
    if (d->n_blobs < 0 || d->n_blobs > GF_MAX_BLOBS || (d->n_blobs > 0 && d->blobs == nullptr)) {
        set_error("gf_medium_create: n_blobs must be in [0, %d] with a table", GF_MAX_BLOBS);
        return GF_ERR_INVALID_ARG;
    }
    if ((d->kind == GF_MED_SPLINE || d->kind == GF_MED_COLD) && d->n_blobs != 0) {
        set_error("gf_medium_create: blobs are only defined for isotropic media");
        return GF_ERR_INVALID_ARG;
    }
    if (d->kind == GF_MED_COLD) {
        if (d->n_species < 1 || d->n_species > GF_MAX_SPECIES) {
            set_error("gf_medium_create: cold plasma needs 1..%d species", GF_MAX_SPECIES);
            return GF_ERR_INVALID_ARG;
        }
        for (int i = 0; i < 2 * d->n_species; ++i)
            if (!std::isfinite(d->species[i])) {
                set_error("gf_medium_create: species values must be finite");
                return GF_ERR_INVALID_ARG;
            }
        for (int i = 0; i < 4; ++i)
            if (!std::isfinite(d->profile[i])) {
                set_error("gf_medium_create: profile values must be finite");
                return GF_ERR_INVALID_ARG;
            }
    } else if (d->n_species != 0) {
        set_error("gf_medium_create: n_species is only defined for GF_MED_COLD");
        return GF_ERR_INVALID_ARG;
    }
    if (d->kind == GF_MED_HOMOG && !(d->n_h > 0 && std::isfinite(d->n_h))) {
        set_error("gf_medium_create: n_h must be a positive finite number");
        return GF_ERR_INVALID_ARG;
    }
    if (d->kind == GF_MED_GRIN && !(std::isfinite(d->n0) && std::isfinite(d->a) && d->n0 > 0)) {
        set_error("gf_medium_create: GRIN needs finite n0 > 0 and a");
        return GF_ERR_INVALID_ARG;
    }
    if (d->kind == GF_MED_SPLINE && (d->grid == nullptr || d->grid_n < 4 || d->grid_n > 2048)) {
        set_error("gf_medium_create: spline needs a grid with 4 <= grid_n <= 2048");
        return GF_ERR_INVALID_ARG;
    }
    // plain rows, then scaled rows (t64); float scaled rows, FP32 pre-test rows and
    // double-float rows (t32)
    const size_t nbl = (size_t)d->n_blobs;
    std::vector<double> t64(2 * kBlobStride * nbl);
    std::vector<float> t32((kBlobStride + 4 + kDfRowFloats) * nbl);
    double pre_span = 0.0;   // max over blobs of sigma, and of sigma |c_i|
    double sig_max = 0.0;
    for (int j = 0; j < d->n_blobs; ++j) {
        const double *b = d->blobs + 5 * j;
        double w = b[4];
        bool fin = std::isfinite(b[0]) && std::isfinite(b[1]) && std::isfinite(b[2]) && std::isfinite(b[3]);
        if (!(w > 0) || !std::isfinite(w) || !fin) {
            set_error("gf_medium_create: blob %d has a non-finite value or width <= 0", j);
            return GF_ERR_INVALID_ARG;
        }
        const double sj = -1.0 / (2.0 * w * w);
        // base-2 scale: A exp(s |x - c|^2) = A 2^(-|u|^2) with u = sig (x - c)
        const double sig = std::sqrt(-sj * kInvLn2);
        if (!(sj < 0) || !std::isfinite(sj) || !(sig > 0) || !std::isfinite(kNeg2Ln2 * sig * b[0])) {
            set_error("gf_medium_create: blob %d: width %g out of range", j, w);
            return GF_ERR_INVALID_ARG;
        }
        const double row[kBlobStride] = {b[0], b[1], b[2], b[3], sj, 2.0 * sj};
        const double srow[kBlobStride] = {sig, -(sig * b[1]), -(sig * b[2]), -(sig * b[3]), b[0],
                                          (kNeg2Ln2 * sig) * b[0]};
        for (int c = 0; c < kBlobStride; ++c) {
            t64[kBlobStride * j + c] = row[c];
            t64[kBlobStride * (nbl + j) + c] = srow[c];
            t32[kBlobStride * j + c] = (float)srow[c];
        }
        for (int c = 0; c < 4; ++c) t32[kBlobStride * nbl + 4 * j + c] = (float)srow[c];
        // double-float row: c_hi[3], c_lo[3], then (hi, lo) of s/ln2, A and 2 s A, with
        // hi = RN_float(v) and lo = RN_float(v - hi) (v - hi is exact in double)
        float *dfr = t32.data() + (kBlobStride + 4) * nbl + kDfRowFloats * j;
        const double vals[6] = {b[1], b[2], b[3], sj * kInvLn2, b[0], (2.0 * sj) * b[0]};
        for (int c = 0; c < 6; ++c) {
            const float hi = (float)vals[c];
            const float lo = (float)(vals[c] - (double)hi);
            const int at = c < 3 ? c : 6 + 2 * (c - 3);
            dfr[at] = hi;
            dfr[c < 3 ? 3 + c : at + 1] = lo;
        }
        sig_max = std::max(sig_max, sig);
        for (int c = 1; c < 4; ++c) pre_span = std::max(pre_span, std::fabs(srow[c]));
    }
    // FP32 pre-test valid while sigma (2 max|x_i| + max|c_i|) <= 1e5 for every blob
    float pre_lim = -1.0f;
    if (d->n_blobs > 0) {
        const double lim = (1e5 - pre_span) / (2.0 * sig_max);
        if (lim > 0) pre_lim = (float)std::min(lim, 1e30);
    }
    gf_medium m = new gf_medium_s();
    cudaGetDevice(&m->device);
    MediumParams &p = m->p;
    p.kind = d->kind;
    p.n_blobs = d->n_blobs;
    p.grid_n = d->grid_n;
    p.pre_lim = pre_lim;
    p.n_h2 = d->n_h * d->n_h;
    p.n02 = d->n0 * d->n0;
    p.n02a2 = d->n0 * d->n0 * d->a * d->a;
    p.n_species = d->kind == GF_MED_COLD ? d->n_species : 0;
    for (int i = 0; i < 2 * GF_MAX_SPECIES; ++i) p.species[i] = i < 2 * p.n_species ? d->species[i] : 0.0;
    for (int i = 0; i < 4; ++i) p.prof[i] = d->kind == GF_MED_COLD ? d->profile[i] : 0.0;
    p.wp_sum = 0.0;
    for (int sp = 0; sp < GF_MAX_SPECIES; ++sp) {
        const bool on = sp < p.n_species;
        p.cold_x[3 * sp] = on ? p.species[2 * sp] * p.prof[1] : 0.0;
        p.cold_x[3 * sp + 1] = on ? p.species[2 * sp + 1] * p.prof[3] : 0.0;
        p.cold_x[3 * sp + 2] = 2.0 * p.cold_x[3 * sp + 1];
        p.wp_sum += on ? p.species[2 * sp] : 0.0;
    }
    gf_status s = GF_OK;
    const size_t n64 = std::max<size_t>(t64.size(), 1), n32 = std::max<size_t>(t32.size(), 1);
    if ((s = cuda_status(dev_alloc(&m->d_blobs64, n64 * sizeof(double)), "cudaMalloc(blobs)")) != GF_OK ||
        (s = cuda_status(dev_alloc(&m->d_blobs32, n32 * sizeof(float)), "cudaMalloc(blobs)")) != GF_OK) {
        free_medium(m);
        return s;
    }
    if (!t64.empty()) {
        if ((s = cuda_status(cudaMemcpy(m->d_blobs64, t64.data(), t64.size() * sizeof(double),
                                        cudaMemcpyHostToDevice), "cudaMemcpy(blobs)")) != GF_OK ||
            (s = cuda_status(cudaMemcpy(m->d_blobs32, t32.data(), t32.size() * sizeof(float),
                                        cudaMemcpyHostToDevice), "cudaMemcpy(blobs)")) != GF_OK) {
            free_medium(m);
            return s;
        }
    }
    p.blobs64 = m->d_blobs64;
    p.blobs32 = m->d_blobs32;
    p.blobs64s = m->d_blobs64 + kBlobStride * nbl;
    p.pre32 = m->d_blobs32 + kBlobStride * nbl;
    p.dfrows = m->d_blobs32 + (kBlobStride + 4) * nbl;
    if (d->kind == GF_MED_SPLINE) {
        size_t nodes = (size_t)d->grid_n * d->grid_n * d->grid_n;
        // finite values only; subnormals (|v| < FLT_MIN) are stored as zero of the same
        // sign (through a flushed host copy, made only when there is one)
        bool subnormal = false;
        for (size_t i = 0; i < nodes * 8; ++i) {
            if (!std::isfinite(d->grid[i])) {
                set_error("gf_medium_create: grid value %zu is not finite", i);
                free_medium(m);
                return GF_ERR_INVALID_ARG;
            }
            subnormal = subnormal || std::fpclassify(d->grid[i]) == FP_SUBNORMAL;
        }
        std::vector<float> flushed;
        if (subnormal) {
            flushed.assign(d->grid, d->grid + nodes * 8);
            for (float &v : flushed)
                if (std::fpclassify(v) == FP_SUBNORMAL) v = std::copysign(0.0f, v);
        }
        const float *src = subnormal ? flushed.data() : d->grid;
        if ((s = cuda_status(dev_alloc(&m->d_grid, nodes * 8 * sizeof(float)), "cudaMalloc(grid)")) != GF_OK ||
            (s = cuda_status(cudaMemcpy(m->d_grid, src, nodes * 8 * sizeof(float),
                                        cudaMemcpyHostToDevice), "cudaMemcpy(grid)")) != GF_OK) {
            free_medium(m);
            return s;
        }
        p.grid = m->d_grid;
    }
    *out = m;
    return GF_OK;
}

gf_status gf_medium_destroy(gf_medium m)
{
    if (m == nullptr) return GF_OK;
    free_medium(m);
    return GF_OK;
}

gf_status gf_medium_set_amplitudes(gf_medium m, const double *amplitudes, void *stream)
{
    gf_status s;
    if ((s = check_medium(m)) != GF_OK) return s;
    if (m->p.n_blobs == 0) {
        set_error("gf_medium_set_amplitudes: medium has no blobs");
        return GF_ERR_INVALID_ARG;
    }
    if ((s = check_device_ptr(amplitudes, "amplitudes")) != GF_OK) return s;
    set_amplitudes_kernel<<<1, GF_MAX_BLOBS, 0, (cudaStream_t)stream>>>(m->d_blobs64, m->d_blobs32,
                                                                        amplitudes, m->p.n_blobs);
    return cuda_status(cudaGetLastError(), "gf_medium_set_amplitudes launch");
}

gf_status gf_rays_onshell(gf_medium m, gf_precision prec, const gf_rays *rays, const void *dir,
                          double omega, void *stream)
{
    gf_status s;
    if ((s = check_medium(m)) != GF_OK) return s;
    if (prec != GF_F32 && prec != GF_F64 && prec != GF_F64X) {
        set_error("gf_rays_onshell: unknown precision %d", (int)prec);
        return GF_ERR_INVALID_ARG;
    }
    if (!(omega > 0) || !std::isfinite(omega)) {
        set_error("gf_rays_onshell: omega must be positive and finite");
        return GF_ERR_INVALID_ARG;
    }
    if (m->p.kind == GF_MED_COLD || m->jit_lib != nullptr) {
        set_error("gf_rays_onshell: not defined for cold-plasma or generated media; use gf_rays_newton_kx");
        return GF_ERR_UNSUPPORTED;
    }
    if ((s = check_rays(rays, false)) != GF_OK) return s;
    if (rays->n == 0) return GF_OK;
    if ((s = check_device_ptr(dir, "dir")) != GF_OK) return s;
    return cuda_status(launch_onshell(m->p, prec, *rays, dir, omega, (cudaStream_t)stream),
                       "gf_rays_onshell launch");
}

gf_status gf_rays_newton_kx(gf_medium m, gf_precision prec, const gf_rays *rays, double omega, double tol,
                            int32_t max_iter, void *stream)
{
    gf_status s;
    if ((s = check_medium(m)) != GF_OK) return s;
    if (prec != GF_F32 && prec != GF_F64 && prec != GF_F64X) {
        set_error("gf_rays_newton_kx: unknown precision %d", (int)prec);
        return GF_ERR_INVALID_ARG;
    }
    if (!(omega > 0) || !std::isfinite(omega) || !(tol > 0) || !std::isfinite(tol) || max_iter < 1 ||
        max_iter > 10000) {
        set_error("gf_rays_newton_kx: need omega > 0, tol > 0, 1 <= max_iter <= 10000");
        return GF_ERR_INVALID_ARG;
    }
    if ((s = check_rays(rays, false)) != GF_OK) return s;
    if (m->jit_lib != nullptr) {
        set_error("gf_rays_newton_kx: not available for generated media");
        return GF_ERR_UNSUPPORTED;
    }
    return cuda_status(launch_newton_kx(m->p, prec, *rays, omega, tol, max_iter, (cudaStream_t)stream),
                       "gf_rays_newton_kx launch");
}

gf_status gf_trace_rk4(gf_medium m, gf_precision prec, const gf_rays *rays, double omega, double dt,
                       int64_t n_steps, double radius, int64_t checkpoint_every, double *ckpt,
                       void *stream)
{
    gf_status s;
    if ((s = check_medium(m)) != GF_OK) return s;
    if (prec != GF_F32 && prec != GF_F64 && prec != GF_F64X) {
        set_error("gf_trace_rk4: unknown precision %d", (int)prec);
        return GF_ERR_INVALID_ARG;
    }
    if (!(omega > 0) || !std::isfinite(omega) || !(dt > 0) || !std::isfinite(dt) || n_steps < 0 ||
        !std::isfinite(radius)) {
        set_error("gf_trace_rk4: need omega > 0, dt > 0, n_steps >= 0, finite radius");
        return GF_ERR_INVALID_ARG;
    }
    if ((s = check_rays(rays, true)) != GF_OK) return s;
    if (m->jit_lib != nullptr) {
        if (prec != GF_F64 || ckpt != nullptr) {
            set_error("gf_trace_rk4: a generated (JIT) medium runs in GF_F64 without checkpoints");
            return GF_ERR_UNSUPPORTED;
        }
        return cuda_status(launch_rk4_jit(m, *rays, omega, dt, n_steps, radius, (cudaStream_t)stream),
                           "gf_trace_rk4 (generated medium) launch");
    }
    if (ckpt != nullptr) {
        if (prec == GF_F32) {
            set_error("gf_trace_rk4: checkpoints are only produced by the FP64 paths");
            return GF_ERR_UNSUPPORTED;
        }
        if (checkpoint_every <= 0) {
            set_error("gf_trace_rk4: checkpoint_every must be > 0 with a checkpoint buffer");
            return GF_ERR_INVALID_ARG;
        }
        if (rays->n > 0 && (s = check_device_ptr(ckpt, "ckpt")) != GF_OK) return s;
    }
    if (rays->n == 0) return GF_OK;
    return cuda_status(launch_rk4(m->p, prec, *rays, omega, dt, n_steps, radius,
                                  ckpt ? checkpoint_every : 1, ckpt, (cudaStream_t)stream),
                       "gf_trace_rk4 launch");
}

gf_status gf_bench_set_counters(unsigned long long *counters)
{
    if (counters && check_device_ptr(counters, "counters") != GF_OK) return GF_ERR_INVALID_ARG;
    g_work_counters = counters;
    return GF_OK;
}

size_t gf_adjoint_scratch_bytes(gf_medium m, int64_t n, int64_t checkpoint_every)
{
    if (m == nullptr || n < 0 || checkpoint_every < 1 || m->p.n_blobs < 1) return 0;
    return adjoint_scratch_bytes(m->p.n_blobs, n, checkpoint_every);
}

gf_status gf_trace_adjoint(gf_medium m, int64_t n, double omega, double dt, int64_t n_steps,
                           int64_t checkpoint_every, const double *ckpt, const int32_t *steps_done,
                           const double *lambda, int64_t ld, double *dL_dtheta, double *dL_dy0,
                           void *scratch, size_t scratch_bytes, void *stream)
{
    gf_status s;
    if ((s = check_medium(m)) != GF_OK) return s;
    if (m->p.kind == GF_MED_SPLINE || m->p.kind == GF_MED_COLD || m->p.n_blobs < 1 || m->jit_lib != nullptr) {
        set_error("gf_trace_adjoint: needs an isotropic medium with at least one blob");
        return GF_ERR_INVALID_ARG;
    }
    if (n < 0 || ld < n || n_steps < 0 || checkpoint_every < 1 || checkpoint_every > 4096 ||
        !(omega > 0) || !std::isfinite(omega) || !(dt > 0) || !std::isfinite(dt)) {
        set_error("gf_trace_adjoint: need n >= 0, ld >= n, n_steps >= 0, 1 <= checkpoint_every <= 4096, "
                  "omega > 0, dt > 0");
        return GF_ERR_INVALID_ARG;
    }
    if ((s = check_device_ptr(dL_dtheta, "dL_dtheta")) != GF_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        return cuda_status(cudaMemsetAsync(dL_dtheta, 0, sizeof(double) * m->p.n_blobs, st),
                           "gf_trace_adjoint memset");
    }
    if ((s = check_device_ptr(ckpt, "ckpt")) != GF_OK || (s = check_device_ptr(steps_done, "steps_done")) != GF_OK ||
        (s = check_device_ptr(lambda, "lambda")) != GF_OK || (s = check_device_ptr(scratch, "scratch")) != GF_OK)
        return s;
    if (dL_dy0 && (s = check_device_ptr(dL_dy0, "dL_dy0")) != GF_OK) return s;
    const size_t need = adjoint_scratch_bytes(m->p.n_blobs, n, checkpoint_every);
    if (scratch_bytes < need) {
        set_error("gf_trace_adjoint: scratch has %zu bytes, needs %zu", scratch_bytes, need);
        return GF_ERR_INVALID_ARG;
    }
    return cuda_status(launch_adjoint(m->p, n, omega, dt, n_steps, checkpoint_every, ckpt, steps_done, lambda,
                                      ld, dL_dtheta, dL_dy0, scratch, st),
                       "gf_trace_adjoint launch");
}

}  // extern "C"
