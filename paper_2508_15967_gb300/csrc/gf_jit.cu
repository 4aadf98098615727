// gf_jit.cu -- run-time compilation of generated dispersion relations.
//
// The symbolic front end (Python, symbolic.py) turns an expression graph of D
// and its chain-rule derivatives into CUDA source for one device function
// (Sec. 2.1-2.2 of the paper: build the graph, differentiate, simplify, emit
// one register per node).  Here that source is compiled together with an RK4
// ray kernel by NVRTC for the current device's architecture (sm_103a on
// GB300) and loaded as a CUDA library; gf_trace_rk4 launches it for media
// created by gf_jit_medium_create.  NVRTC is loaded with dlopen on first use,
// so the library itself does not depend on it.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "gf_internal.cuh"

namespace gf {

// Table-driven exponential available to generated code as gf_exp(a) of a
// natural-base argument of either sign: Tang's method with the library's
// 2^(j/2048) table (staged in shared memory by the kernel below), a
// Cody-Waite two-part reduction by ln2/2048 and a degree-3 polynomial,
// < 1.35 ulp, for |a| < 708; CUDA's exp outside (overflow, underflow, inf,
// NaN).  The table and constants are printed into the source as exact hex
// literals.
static const char *kJitExp = R"JIT(
__shared__ double gf_T[2048];
__device__ __forceinline__ double gf_exp(double a)
{
    const unsigned ahi = (unsigned)__double2hiint(a) & 0x7fffffffu;
    if (ahi >= 0x40862000u) return exp(a);           // |a| >= 708, inf, NaN
    const double shifter = 6755399441055744.0;
    const double t = fma(a, GF_INV_LN2_N, shifter);
    const int k = __double2loint(t);
    const double kd = t - shifter;
    double r = fma(kd, -GF_LN2_N_HI, a);
    r = fma(kd, -GF_LN2_N_LO, r);
    const double c = fma(r, 1.0 / 6.0, 0.5);
    const double p = fma(r * r, c, r);
    const double Tj = gf_T[k & 2047];
    const double v = fma(Tj, p, Tj);
    return __hiloint2double(__double2hiint(v) + ((k >> 11) << 20), __double2loint(v));
}
)JIT";

static const double kHostExpTab[kExpTabN] = {GF_EXP2_TAB_VALUES};

// The exp table as a device array initialiser plus the reduction constants.
static const std::string &jit_prelude()
{
    static const std::string text = [] {
        std::string t;
        char buf[64];
        snprintf(buf, sizeof buf, "#define GF_INV_LN2_N %a\n", kInvLn2xN);
        t += buf;
        snprintf(buf, sizeof buf, "#define GF_LN2_N_HI %a\n", kLn2ByNHi);
        t += buf;
        snprintf(buf, sizeof buf, "#define GF_LN2_N_LO %a\n", kLn2ByNLo);
        t += buf;
        t += "__device__ const double gf_exp2_tab[2048] = {\n";
        for (int j = 0; j < kExpTabN; ++j) {
            snprintf(buf, sizeof buf, "%a,%s", kHostExpTab[j], (j % 4 == 3) ? "\n" : " ");
            t += buf;
        }
        t += "};\n";
        t += kJitExp;
        return t;
    }();
    return text;
}

// RK4 ray kernel around the generated gf_user_dispersion(y, w, out):
// out = (D, D_x0, D_x1, D_x2, D_k0, D_k1, D_k2, D_w).  Same update, statuses
// and residual bookkeeping as the built-in kernel; the right-hand side is the
// generic f = (-D_k / D_w, D_x / D_w) and a cut-off is D_w = 0.
static const char *kJitKernel = R"JIT(
__device__ __forceinline__ bool gf_rhs(const double *y, double w, double *f, double *D)
{
    double o[8];
    gf_user_dispersion(y, w, o);
    *D = o[0];
    const double dw = o[7];
    if (!(dw != 0.0) || !isfinite(dw)) return false;
    const double inv = 1.0 / dw;
    f[0] = -o[4] * inv; f[1] = -o[5] * inv; f[2] = -o[6] * inv;
    f[3] = o[1] * inv;  f[4] = o[2] * inv;  f[5] = o[3] * inv;
    return true;
}

extern "C" __global__ void __launch_bounds__(128) gf_jit_rk4(
    long long n, long long ld, double *y, double *t, int *status, int *steps, double *dres,
    double *dmax, double w, double dt, long long n_steps, double r2)
{
    for (int j = threadIdx.x; j < 2048; j += blockDim.x) gf_T[j] = gf_exp2_tab[j];
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || status[i] != 0) return;
    double s[6];
    for (int c = 0; c < 6; ++c) s[c] = y[c * ld + i];
    double dm = dmax ? dmax[i] : 0.0;
    int st = 0;
    long long k = 0;
    const double h2 = 0.5 * dt, h6 = dt / 6.0;
    for (; k < n_steps; ++k) {
        double K[6], acc[6], Y[6], D, Dd;
        bool ok = gf_rhs(s, w, K, &D);
        dm = fmax(dm, fabs(D));
        if (!ok) { st = 2; break; }
        for (int c = 0; c < 6; ++c) { acc[c] = K[c]; Y[c] = s[c] + h2 * K[c]; }
        if (!gf_rhs(Y, w, K, &Dd)) { st = 2; break; }
        for (int c = 0; c < 6; ++c) { acc[c] += 2.0 * K[c]; Y[c] = s[c] + h2 * K[c]; }
        if (!gf_rhs(Y, w, K, &Dd)) { st = 2; break; }
        for (int c = 0; c < 6; ++c) { acc[c] += 2.0 * K[c]; Y[c] = s[c] + dt * K[c]; }
        if (!gf_rhs(Y, w, K, &Dd)) { st = 2; break; }
        double yn[6];
        bool fin = true;
        for (int c = 0; c < 6; ++c) { yn[c] = s[c] + h6 * (acc[c] + K[c]); fin = fin && isfinite(yn[c]); }
        if (!fin) { st = 3; break; }
        for (int c = 0; c < 6; ++c) s[c] = yn[c];
        if (r2 > 0.0 && s[0] * s[0] + s[1] * s[1] + s[2] * s[2] > r2) { st = 1; ++k; break; }
    }
    double K[6], D;
    gf_rhs(s, w, K, &D);
    dm = fmax(dm, fabs(D));
    if (dres) dres[i] = fabs(D);
    if (dmax) dmax[i] = dm;
    for (int c = 0; c < 6; ++c) y[c * ld + i] = s[c];
    if (k > 0) t[i] = __dadd_rn(t[i], __dmul_rn((double)k, dt));
    steps[i] += (int)k;
    status[i] = st;
}
)JIT";

struct Nvrtc {
    void *h = nullptr;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcGetErrorString) err = nullptr;
};

static std::mutex g_nvrtc_mutex;
static Nvrtc g_nvrtc;

static gf_status load_nvrtc(Nvrtc **out)
{
    std::lock_guard<std::mutex> lock(g_nvrtc_mutex);
    if (g_nvrtc.h == nullptr) {
        const char *names[] = {"libnvrtc.so.13", "/usr/local/cuda/lib64/libnvrtc.so.13", "libnvrtc.so"};
        for (const char *n : names)
            if ((g_nvrtc.h = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (g_nvrtc.h == nullptr) {
            set_error("NVRTC (libnvrtc.so.13) could not be loaded: %s", dlerror());
            return GF_ERR_UNSUPPORTED;
        }
#define GF_SYM(f, s) g_nvrtc.f = (decltype(g_nvrtc.f))dlsym(g_nvrtc.h, s)
        GF_SYM(create, "nvrtcCreateProgram");
        GF_SYM(compile, "nvrtcCompileProgram");
        GF_SYM(log_size, "nvrtcGetProgramLogSize");
        GF_SYM(log, "nvrtcGetProgramLog");
        GF_SYM(cubin_size, "nvrtcGetCUBINSize");
        GF_SYM(cubin, "nvrtcGetCUBIN");
        GF_SYM(destroy, "nvrtcDestroyProgram");
        GF_SYM(err, "nvrtcGetErrorString");
#undef GF_SYM
        if (!g_nvrtc.create || !g_nvrtc.compile || !g_nvrtc.log_size || !g_nvrtc.log || !g_nvrtc.cubin_size ||
            !g_nvrtc.cubin || !g_nvrtc.destroy || !g_nvrtc.err) {
            set_error("NVRTC is missing an entry point");
            dlclose(g_nvrtc.h);
            g_nvrtc = Nvrtc{};
            return GF_ERR_UNSUPPORTED;
        }
    }
    *out = &g_nvrtc;
    return GF_OK;
}

// Compile generated source + the kernel template to a cubin for `arch`.
static gf_status compile(const char *source, const char *arch, std::vector<char> &cubin, std::string &log)
{
    Nvrtc *nv = nullptr;
    gf_status s = load_nvrtc(&nv);
    if (s != GF_OK) return s;
    const std::string full = jit_prelude() + std::string(source) + "\n" + kJitKernel;
    nvrtcProgram prog;
    nvrtcResult r = nv->create(&prog, full.c_str(), "gf_generated_medium.cu", 0, nullptr, nullptr);
    if (r != NVRTC_SUCCESS) {
        set_error("nvrtcCreateProgram: %s", nv->err(r));
        return GF_ERR_CUDA;
    }
    const std::string arch_opt = std::string("-arch=") + arch;
    const char *opts[] = {arch_opt.c_str(), "--std=c++17", "-default-device", "-lineinfo"};
    r = nv->compile(prog, 4, opts);
    size_t n = 0;
    nv->log_size(prog, &n);
    log.assign(n ? n - 1 : 0, '\0');
    if (n > 1) nv->log(prog, &log[0]);
    if (r != NVRTC_SUCCESS) {
        set_error("generated medium does not compile: %s", log.substr(0, 400).c_str());
        nv->destroy(&prog);
        return GF_ERR_INVALID_ARG;
    }
    size_t cs = 0;
    nv->cubin_size(prog, &cs);
    cubin.resize(cs);
    r = nv->cubin(prog, cubin.data());
    nv->destroy(&prog);
    if (r != NVRTC_SUCCESS || cs == 0) {
        set_error("nvrtcGetCUBIN failed");
        return GF_ERR_CUDA;
    }
    return GF_OK;
}

cudaError_t launch_rk4_jit(gf_medium m, const gf_rays &r, double omega, double dt, int64_t n_steps,
                           double radius, cudaStream_t s)
{
    if (r.n == 0) return cudaSuccess;
    long long n = r.n, ld = r.ld, ns = n_steps;
    double w = omega, h = dt, r2 = radius > 0 ? radius * radius : 0.0;
    void *y = r.y;
    double *t = r.t, *dres = r.d_res, *dmax = r.d_max;
    int32_t *status = r.status, *steps = r.steps;
    void *args[] = {&n, &ld, &y, &t, &status, &steps, &dres, &dmax, &w, &h, &ns, &r2};
    const unsigned blocks = (unsigned)((r.n + 127) / 128);
    return cudaLaunchKernel((const void *)m->jit_kernel, dim3(blocks), dim3(128), args, 0, s);
}

}  // namespace gf

using namespace gf;

extern "C" {

gf_status gf_jit_compile_check(const char *source, const char *arch, char *log, size_t log_size)
{
    if (source == nullptr || arch == nullptr) {
        set_error("gf_jit_compile_check: source and arch must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    std::vector<char> cubin;
    std::string lg;
    gf_status s = compile(source, arch, cubin, lg);
    if (log && log_size) {
        snprintf(log, log_size, "%s", lg.c_str());
    }
    return s;
}

gf_status gf_jit_medium_create(const char *source, gf_medium *out)
{
    if (source == nullptr || out == nullptr) {
        set_error("gf_jit_medium_create: source and out must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int dev = 0, major = 0, minor = 0;
    gf_status s;
    if ((s = cuda_status(cudaGetDevice(&dev), "cudaGetDevice")) != GF_OK) return s;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    char arch[32];
    snprintf(arch, sizeof arch, "sm_%d%da", major, minor);
    std::vector<char> cubin;
    std::string log;
    if ((s = compile(source, arch, cubin, log)) != GF_OK) return s;
    gf_medium m = new gf_medium_s();
    m->device = dev;
    m->p.kind = -1;
    if ((s = cuda_status(cudaLibraryLoadData(&m->jit_lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0),
                         "cudaLibraryLoadData")) != GF_OK ||
        (s = cuda_status(cudaLibraryGetKernel(&m->jit_kernel, m->jit_lib, "gf_jit_rk4"),
                         "cudaLibraryGetKernel")) != GF_OK) {
        if (m->jit_lib) cudaLibraryUnload(m->jit_lib);
        delete m;
        return s;
    }
    *out = m;
    return GF_OK;
}

}  // extern "C"
