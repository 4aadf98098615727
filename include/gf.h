/*
 * gf.h -- C ABI of the GB300 Hamiltonian ray-tracing library (libgf.so).
 *
 * The library advances many independent rays of a wave whose dispersion
 * relation is D(x, k, w) = 0 (arXiv 2508.15967, Sec. 4).  Along a ray D is
 * constant (Eq. 1) and the equations actually integrated come from implicit
 * differentiation (Eqs. 2-3):
 *
 *     dx/dt =  dw/dk = -D_k / D_w,        dk/dt = -dw/dx = D_x / D_w.
 *
 * Supported media (D and its gradients are hand-derived and fused on device):
 *   GF_MED_HOMOG      D = |k|^2 - w^2 n_h^2
 *   GF_MED_LUNEBURG   D = |k|^2 - w^2 n^2(x),  n^2 = 2 - |x|^2 for |x|^2 <= 1, else 1
 *   GF_MED_GRIN       D = |k|^2 - w^2 n^2(x),  n^2 = n0^2 (1 - a^2 (y^2 + z^2))
 *   GF_MED_QUADRATIC  D = |k|^2 - w^2 (2 - |x|^2)        (Luneburg law, no kink)
 *   GF_MED_SPLINE     D = k^T M(x) k - w^2 eps(x), M (symmetric 3x3) and eps from
 *                     a periodic tricubic B-spline grid on [-1, 1)^3
 *   GF_MED_COLD       cold magnetised plasma, D = det(eps + n n - n^2 I), n = k/w
 *                     (c = 1), B along z, slab profiles along x (Sec. 4.1, Eqs. 4-10)
 * Every isotropic medium may add Gaussian blobs to n^2:
 *   n^2 += sum_j A_j exp(-|x - c_j|^2 / (2 w_j^2)).
 *
 * Conventions for every entry point:
 *   - Device pointers are caller-owned CUDA global memory on the current
 *     device (for example torch tensors); the library never frees them.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and returns without synchronising, unless stated.
 *   - The return value is a gf_status; GF_OK on success.  On failure a
 *     description is available from gf_last_error() (thread-local).  Argument
 *     errors are detected on the host before anything is enqueued.
 *   - Per-ray outcomes (exit, cut-off, ...) are ray statuses, not call errors.
 *   - Nothing traps: device-side failures are reported through statuses.
 *
 * Ray state layout (struct gf_rays): structure of arrays, component c of ray
 * i at y[c * ld + i] with c = 0..5 = (x, y, z, kx, ky, kz).  A sub-range of a
 * larger ray set is addressed by offsetting every pointer and keeping ld.
 */
#ifndef GF_H
#define GF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GF_OK = 0,
    GF_ERR_INVALID_ARG = 1,   /* a NULL required pointer, a bad size or value       */
    GF_ERR_CUDA = 2,          /* a CUDA runtime call failed (text in gf_last_error) */
    GF_ERR_OOM = 3,           /* device memory allocation failed                    */
    GF_ERR_UNSUPPORTED = 4,   /* valid request the library does not provide         */
    GF_ERR_TIMEOUT = 5        /* a bounded device-side wait gave up                 */
} gf_status;

/* GF_F64: every operation in IEEE double.  GF_F32: float, Kahan-compensated
 * state.  GF_F64X: double state, integrator, D and right-hand side, with the
 * Gaussian-blob sums computed in double-float (pairs of floats, ~48-bit
 * significand, relative error ~1e-15 per term) on the FP32 pipes; ray buffers
 * as for GF_F64. */
typedef enum { GF_F32 = 0, GF_F64 = 1, GF_F64X = 2 } gf_precision;

typedef enum {
    GF_MED_HOMOG = 0,
    GF_MED_LUNEBURG = 1,
    GF_MED_GRIN = 2,
    GF_MED_QUADRATIC = 3,
    GF_MED_SPLINE = 4,
    GF_MED_COLD = 5
} gf_medium_kind;

/* Ray status codes, stored per ray (int32). */
enum {
    GF_RAY_ACTIVE = 0,          /* still propagating; another call continues it        */
    GF_RAY_EXITED = 1,          /* a step ended outside the termination sphere          */
    GF_RAY_CUTOFF = 2,          /* reached n^2 <= 0 (eps <= 0), i.e. D_w = 0: cut-off  */
    GF_RAY_NONFINITE = 3,       /* an update was inf/nan; the state before it is kept  */
    GF_RAY_MAX_STEPS = 4,       /* adaptive stepping used its step budget              */
    GF_RAY_STEP_UNDERFLOW = 5,  /* adaptive step fell below 1e-14 max(1, |t|)          */
    GF_RAY_DONE = 6             /* adaptive stepping reached t_max                     */
};

#define GF_MAX_BLOBS 64         /* blobs per medium                                   */
#define GF_MAX_SPECIES 4        /* cold-plasma species                                */

/* Host-side description of a medium, read only during gf_medium_create. */
typedef struct {
    int32_t kind;               /* gf_medium_kind                                        */
    int32_t n_blobs;            /* 0..GF_MAX_BLOBS; isotropic media only                  */
    int32_t grid_n;             /* GF_MED_SPLINE: nodes per axis (>= 4)                   */
    int32_t reserved;           /* must be 0                                              */
    double n_h;                 /* GF_MED_HOMOG: refractive index (> 0)                   */
    double n0, a;               /* GF_MED_GRIN: axis index and gradient constant          */
    const double *blobs;        /* host, n_blobs rows (A, cx, cy, cz, w), w > 0           */
    const float *grid;          /* host, grid_n^3 nodes x 8 floats, x fastest, node
                                   (ix, iy, iz) at (-1 + ix h, ...), h = 2 / grid_n, holding
                                   (M11, M12, M13, M22, M23, M33, eps, unused); the values
                                   are B-spline control coefficients (no prefilter), all
                                   finite; subnormal values are read as zero              */
    /* GF_MED_COLD: species s has squared plasma frequency w_p,s^2 f(x) and signed
       cyclotron frequency Omega_s g(x), with f(x) = profile[0] + profile[1] x_0 (the
       density, e.g. the linear gradient 0.1 x + 1 of Eq. 4) and g(x) = profile[2] +
       profile[3] x_0 (|B|).  S = 1 - sum w_p^2/(w^2 - Omega^2),
       Dst = sum Omega w_p^2/(w (w^2 - Omega^2)), P = 1 - sum w_p^2/w^2 (Eqs. 7-10);
       with a = n_x^2 + n_y^2, b = n_z^2:
       D = S a (a+b) + P b (a+b) - (S^2 - Dst^2) a - P S (a+2b) + P (S^2 - Dst^2). */
    int32_t n_species;          /* 1..GF_MAX_SPECIES for GF_MED_COLD, else 0              */
    int32_t reserved2;          /* must be 0                                              */
    double species[2 * GF_MAX_SPECIES];   /* (w_p,s^2, Omega_s) pairs                     */
    double profile[4];          /* f0, f1, g0, g1                                         */
} gf_medium_desc;

typedef struct gf_medium_s *gf_medium;

/* Ray buffers, all device memory, caller-owned. */
typedef struct {
    int64_t n;                  /* number of rays (0 allowed: the call does nothing)     */
    int64_t ld;                 /* stride between the 6 state rows, >= n                  */
    void *y;                    /* 6 x ld: double for GF_F64, float for GF_F32            */
    double *t;                  /* n: time of each ray                                    */
    int32_t *status;            /* n: GF_RAY_*; only GF_RAY_ACTIVE rays are advanced      */
    int32_t *steps;             /* n: steps taken, incremented by every accepted step     */
    double *d_res;              /* n or NULL: |D| at the final state                      */
    double *d_max;              /* n or NULL: running max of |D| over every state visited */
} gf_rays;

/* Adaptive step control for gf_trace_dopri5. */
typedef struct {
    double rtol, atol;          /* error tolerances (> 0)                                */
    double h0;                  /* first trial step (> 0)                                */
    double t_max;               /* stop (GF_RAY_DONE) at this time                       */
    double radius;              /* stop (GF_RAY_EXITED) outside |x| = radius; <= 0: none */
    double fac_min, fac_max;    /* step-ratio clamps, 0 < fac_min < 1 < fac_max          */
    double safety;              /* controller safety factor, (0, 1]                      */
    int64_t max_steps;          /* accepted-step budget per ray (> 0)                    */
} gf_step_ctl;

/* Text of the last error on this thread ("" if none).  Never NULL. */
const char *gf_last_error(void);

/* Library version as an integer, major * 10000 + minor * 100 + patch. */
int32_t gf_version(void);

/*
 * gf_medium_create -- copy a medium description to the current device.
 * Paper: the dispersion relation and its spatial dependence through the
 * medium (Sec. 4); the spline grid is the counterpart of the paper's
 * argument-dependent coefficient nodes used for spline interpolation (Sec. 2.1).
 * desc: host description (read during the call only).  out: receives a handle
 * owned by the caller until gf_medium_destroy.  Synchronous (blocking copy).
 * Errors: GF_ERR_INVALID_ARG (unknown kind, n_blobs out of range, non-positive
 * width or index, missing grid, non-finite grid value, reserved != 0),
 * GF_ERR_OOM, GF_ERR_CUDA.
 */
gf_status gf_medium_create(const gf_medium_desc *desc, gf_medium *out);

/* gf_medium_destroy -- free the device copy of a medium (NULL: no-op).  Blocks
 * until the device is done with it. */
gf_status gf_medium_destroy(gf_medium m);

/*
 * gf_medium_set_amplitudes -- replace the blob amplitudes A_j (the parameters
 * theta of the adjoint problem) from n_blobs device doubles, stream-ordered.
 * Errors: GF_ERR_INVALID_ARG (NULL, medium without blobs), GF_ERR_CUDA.
 */
gf_status gf_medium_set_amplitudes(gf_medium m, const double *amplitudes, void *stream);

/*
 * gf_rays_onshell -- set k = s d with s > 0 so that D(x, s d, w) = 0 at every
 * ray's current position x (rows 0..2 of rays->y).
 * Paper: initial conditions fix w and x and solve D = 0 for the remaining
 * wave-vector freedom (Sec. 4, to |D| < 1e-15).  Along a fixed direction both
 * media are quadratic in s, so s = w sqrt(eps / q) in closed form, with
 * q = d.d (isotropic) or d^T M d (spline), eps = n^2 or eps.
 * dir: device, 3 rows of rays->ld elements (same type as y), need not be unit.
 * Writes rows 3..5 of y; status = GF_RAY_CUTOFF and k = 0 where eps <= 0 or
 * q <= 0, else GF_RAY_ACTIVE.  Leaves t, steps, d_res, d_max untouched.
 * Errors: GF_ERR_INVALID_ARG, GF_ERR_UNSUPPORTED (GF_MED_COLD: two branches,
 * use gf_rays_newton_kx with a guess that selects one), GF_ERR_CUDA.
 */
gf_status gf_rays_onshell(gf_medium m, gf_precision prec, const gf_rays *rays, const void *dir,
                          double omega, void *stream);

/*
 * gf_rays_newton_kx -- the paper's ray initialisation (Sec. 4): with w, x, k_y
 * and k_z fixed, solve D(x, k, w) = 0 for k_x by Newton's method,
 * k_x <- k_x - D / (dD/dk_x), to |D| < tol (the paper uses 1e-15); the k_x in
 * rays->y on entry is the initial guess and selects the root (D is quadratic
 * in k_x for every medium here, so the guess picks one of two branches).  An
 * iteration whose step no longer changes k_x beyond rounding (|dk_x| <=
 * 2^-50 |k_x|) ends the solve, converged if |D| <= 8 tol.  Writes row 3 of y
 * and status: GF_RAY_ACTIVE when converged, GF_RAY_CUTOFF when no real root
 * was reached in max_iter iterations (evanescent: k_y, k_z too large) or
 * dD/dk_x vanished; leaves t, steps, d_res, d_max untouched.
 * Errors: GF_ERR_INVALID_ARG (tol <= 0, max_iter outside [1, 10000], ...),
 * GF_ERR_CUDA.
 */
gf_status gf_rays_newton_kx(gf_medium m, gf_precision prec, const gf_rays *rays, double omega, double tol,
                            int32_t max_iter, void *stream);

/*
 * gf_trace_rk4 -- advance every active ray by up to n_steps classic RK4 steps
 * of fixed size dt of the ray equations (Eqs. 2-3), fused into one kernel with
 * the ray state held in registers (Sec. 4: one kernel with inputs x, k, t, w
 * and outputs the updated x, k, t and the dispersion residual).
 * Per step: K1 = f(y), K2 = f(y + dt/2 K1), K3 = f(y + dt/2 K2),
 * K4 = f(y + dt K3), y <- y + dt/6 (K1 + 2 K2 + 2 K3 + K4), t = t_0 + n dt.
 * A ray stops early with GF_RAY_CUTOFF (a stage point with eps <= 0, or
 * D_w = 0 for a cold plasma; state kept before that step), GF_RAY_NONFINITE, or GF_RAY_EXITED (a step ending
 * with |x| > radius, radius > 0).  d_max (if given) becomes max(d_max, |D|)
 * over the states visited; d_res (if given) = |D| at the final state.
 * omega > 0; dt > 0; n_steps >= 0.
 * ckpt (GF_F64 only, may be NULL): device doubles [n_ckpt][6][rays->n] with
 * n_ckpt = ceil(n_steps / checkpoint_every); slot j receives the state before
 * step j * checkpoint_every of this call (rays that stopped earlier leave
 * their later slots unwritten).
 * prec: GF_F64 computes in double; GF_F32 in float with Kahan-compensated
 * state updates, t kept in double; GF_F64X as GF_F64 with the blob sums in
 * double-float (media without blobs run the GF_F64 kernel).
 * Errors: GF_ERR_INVALID_ARG, GF_ERR_UNSUPPORTED (ckpt with GF_F32),
 * GF_ERR_CUDA.  gf_rays_onshell and gf_rays_newton_kx treat GF_F64X as GF_F64.
 */
gf_status gf_trace_rk4(gf_medium m, gf_precision prec, const gf_rays *rays, double omega,
                       double dt, int64_t n_steps, double radius, int64_t checkpoint_every,
                       double *ckpt, void *stream);

/* ------------------------------------------------------- generated media */

/*
 * gf_jit_medium_create -- compile a generated dispersion relation into an RK4
 * ray kernel at run time and wrap it as a medium for gf_trace_rk4.
 * Paper: expression graphs of D are differentiated and simplified
 * symbolically, then emitted as kernel source -- one register per node, each
 * shared sub-graph once -- and JIT-compiled for the device (Sec. 2.1-2.2);
 * the RK4 ray update is one fused kernel (Sec. 4).
 * source: CUDA C defining
 *   __device__ void gf_user_dispersion(const double *y, double w, double *out)
 * with y = (x0, x1, x2, k0, k1, k2) and out[0..7] = (D, D_x0, D_x1, D_x2,
 * D_k0, D_k1, D_k2, D_w) (the symbolic front end writes it).  The source may
 * call double gf_exp(double), the library's table-driven exponential (error
 * < 1.35 ulp for |a| < 708, CUDA's exp outside).  It is compiled
 * with NVRTC (loaded on first use) for the current device (sm_103a on GB300)
 * together with the library's RK4 kernel; the right-hand side is the generic
 * f = (-D_k / D_w, D_x / D_w) and a ray stops with GF_RAY_CUTOFF where D_w = 0
 * or is not finite.  Such a medium runs in gf_trace_rk4 with GF_F64 only,
 * without checkpoints; destroy it with gf_medium_destroy.  Synchronous.
 * Errors: GF_ERR_INVALID_ARG (the source does not compile; the compiler log
 * is in gf_last_error), GF_ERR_UNSUPPORTED (NVRTC not available), GF_ERR_CUDA.
 */
gf_status gf_jit_medium_create(const char *source, gf_medium *out);

/*
 * gf_jit_compile_check -- compile generated source for `arch` (e.g. "sm_103a")
 * without loading it (no device needed); the NVRTC log is copied to `log`
 * (may be NULL, truncated to log_size).  Errors as gf_jit_medium_create.
 */
gf_status gf_jit_compile_check(const char *source, const char *arch, char *log, size_t log_size);

/* ------------------------------------------------------------------ adjoint */

/*
 * gf_adjoint_scratch_bytes -- bytes of device scratch gf_trace_adjoint needs
 * for n rays, the medium's blob count and segments of checkpoint_every steps:
 * 8 * (n_blobs * n + checkpoint_every * 4 * 10 * n) + 256 (the parameter
 * gradient of every ray, then the point, n^2 and grad n^2 of every stage of
 * one segment; 1.38 GB for 65,536 rays, 64 blobs and checkpoints every 64
 * steps).  Returns 0 for invalid arguments.
 */
size_t gf_adjoint_scratch_bytes(gf_medium m, int64_t n, int64_t checkpoint_every);

/*
 * gf_trace_adjoint -- gradient of a scalar loss L(y_N) with respect to the blob
 * amplitudes theta_j = A_j of an isotropic medium, by the discrete adjoint of
 * the fixed-step RK4 trace of gf_trace_rk4 (the ray equations of Eqs. 2-3
 * under the RK4 update of Sec. 4; the paper differentiates its expressions
 * symbolically, Sec. 2.1, here the reverse sweep is hand-derived).
 * For every step, backwards, with stage points Y_i and lambda = dL/dy_{n+1}:
 * Kbar_i = dt b_i lambda + dt a_{i+1} Ybar_{i+1}, Ybar_i = J_f(Y_i)^T Kbar_i,
 * thetabar += (df/dtheta)(Y_i)^T Kbar_i, lambda <- lambda + sum_i Ybar_i.
 * Inputs (device): ckpt [n_ckpt][6][n] doubles written by gf_trace_rk4 with
 * the same checkpoint_every (n_ckpt = ceil(n_steps / checkpoint_every));
 * steps_done [n] int32, the steps that forward call applied to each ray (a
 * ray that stopped early is differentiated through the steps it took; stop
 * decisions are held fixed); lambda [6][ld] doubles, dL/dy_N.  Outputs
 * (device): dL_dtheta [n_blobs] doubles, overwritten; dL_dy0 [6][ld] or NULL.
 * scratch: device, >= gf_adjoint_scratch_bytes(m, n, checkpoint_every) bytes,
 * contents overwritten.  The medium must hold the amplitudes of the forward
 * trace.  Each segment is recomputed from its checkpoint with the forward
 * kernel's arithmetic (the recomputed states are the forward trace's bits);
 * the blob terms of the reverse sweep are evaluated in double-float (float
 * pairs, ~48-bit significands; relative error ~1e-14 in the derivative
 * factors).  Deterministic (per-ray accumulators updated in program order,
 * fixed-order reductions), and independent of checkpoint_every bit for bit.
 * Errors: GF_ERR_INVALID_ARG (no blobs, spline medium, bad sizes, small
 * scratch, non-device pointers), GF_ERR_CUDA.
 */
gf_status gf_trace_adjoint(gf_medium m, int64_t n, double omega, double dt, int64_t n_steps,
                           int64_t checkpoint_every, const double *ckpt, const int32_t *steps_done,
                           const double *lambda, int64_t ld, double *dL_dtheta, double *dL_dy0,
                           void *scratch, size_t scratch_bytes, void *stream);

/*
 * gf_trace_adjoint_static -- gf_trace_adjoint without a scratch argument and
 * without any device allocation, for callers that cannot allocate device
 * memory once they are running: for example a real-time experiment-control
 * loop that needs gradients between shots, where cudaMalloc and cudaFree can
 * block or implicitly synchronise the whole device and break the loop's
 * timing, or a host code whose device memory is reserved up front by its own
 * pool.  The paper has no counterpart; this is a deployment variant.
 * Same arguments, layouts, result and errors as gf_trace_adjoint (identical
 * kernels, so bit-identical results), except that the scratch is a fixed
 * 64 MiB device array inside the library: calls needing more than
 * gf_adjoint_scratch_bytes(m, n, checkpoint_every) <= 64 MiB (about 3,190
 * rays with 64 blobs and checkpoints every 64 steps, 11,900 with checkpoints
 * every 16) fail with GF_ERR_INVALID_ARG before anything is enqueued.  The
 * array is held by every GPU on which the library's adjoint module is loaded,
 * until the process exits.  Every call looks up the array's device address
 * in the current context (cudaGetSymbolAddress; nothing is cached, so a
 * context created anew after a device reset is handled).  Under CUDA's lazy
 * module loading the first call on a device may itself load the module and
 * map the 64 MiB, which can block or synchronise the device: make one
 * warm-up call per device before the time-critical loop and before any
 * stream capture (n = 0 serves: it loads the module, sets dL_dtheta to zero
 * and launches nothing else).  All calls share the one array: calls whose
 * work overlaps on the GPU (different streams, or different threads on the
 * same device) race on it and must be serialised by the caller.  The call
 * zeroes what must start at zero (the per-ray gradient accumulators) itself;
 * every other word it reads is written earlier in the same call.
 */
gf_status gf_trace_adjoint_static(gf_medium m, int64_t n, double omega, double dt, int64_t n_steps,
                                  int64_t checkpoint_every, const double *ckpt, const int32_t *steps_done,
                                  const double *lambda, int64_t ld, double *dL_dtheta, double *dL_dy0,
                                  void *stream);

/* ------------------------------------------------------------ batched DOPRI5 */

/* A batch of media whose rays are stored contiguously per medium. */
typedef struct gf_batch_s *gf_batch;

typedef enum {
    GF_SCHED_PERSISTENT = 0,    /* one persistent work-stealing launch (CUDA graph)     */
    GF_SCHED_PER_MEDIUM = 1     /* one launch per medium (CUDA graph of n_media launches) */
} gf_schedule;

/* Launch shape of the persistent schedule (see gf_dopri5_autotune). */
typedef struct {
    int32_t block;              /* threads per block: 64, 128 or 256                     */
    int32_t rays_per_thread;    /* ray slots interleaved per thread: 1 or 2              */
    int32_t compaction;         /* attempted steps between refills of finished lanes     */
    int32_t chunk;              /* rays per work item popped from the queue (>= 1)       */
} gf_tune;

#define GF_MAX_BATCH_BLOBS 16   /* blobs per medium in a batch                         */

/*
 * gf_batch_create -- gather n_media isotropic media of one kind, each with at
 * most GF_MAX_BATCH_BLOBS blobs, into one device table; the rays of medium j
 * are rays [offsets[j], offsets[j+1]) of the ray buffers later passed to
 * gf_trace_dopri5.  offsets: host, n_media + 1 non-decreasing int64, offsets[0]
 * >= 0.  The media may be destroyed afterwards (the batch holds copies).
 * Synchronous.  Errors: GF_ERR_INVALID_ARG (NULL, n_media < 1, mixed kinds,
 * spline media, too many blobs, bad offsets), GF_ERR_OOM, GF_ERR_CUDA.
 */
gf_status gf_batch_create(const gf_medium *media, int32_t n_media, const int64_t *offsets,
                          gf_batch *out);

/* gf_batch_destroy -- free a batch and its cached CUDA graphs (NULL: no-op). */
gf_status gf_batch_destroy(gf_batch b);

/*
 * gf_trace_dopri5 -- trace every active ray of the batch with adaptive
 * Dormand-Prince 5(4) steps until it stops: GF_RAY_EXITED (an accepted step
 * ending outside |x| = ctl->radius; no event location), GF_RAY_DONE (t reached
 * ctl->t_max, the last step shortened to land on it), GF_RAY_MAX_STEPS,
 * GF_RAY_STEP_UNDERFLOW, GF_RAY_CUTOFF or GF_RAY_NONFINITE.
 * Paper: the ray equations of Eqs. 2-3 (the paper integrates them with RK4;
 * the embedded 5(4) pair, its error norm and step controller follow Dormand &
 * Prince 1980 and Hairer-Norsett-Wanner I, Sec. II.4): err = RMS over the 6
 * components of e_i / (atol + rtol max(|y_i|, |y_new,i|)), accept iff err <= 1,
 * h <- h min(fac_max, max(fac_min, safety err^(-1/5))), no growth on the step
 * after a rejection (the norm and the step factor are evaluated in FP32 from
 * the FP64 estimate e).  The blob sums are IEEE double, or double-float after
 * gf_batch_set_precision(b, GF_F64X).  rays->steps counts accepted steps; rejects (device, n,
 * may be NULL) counts rejected ones.  Every ray starts from h = ctl->h0.
 * Results of a ray do not depend on the schedule: both schedules return bit-
 * identical buffers.  sched selects the launch structure; tune (may be NULL:
 * defaults, or the last gf_dopri5_autotune result of this batch) shapes the
 * persistent launch.  The first call with a given argument set captures a
 * CUDA graph on a private stream and later calls replay it on `stream`.
 * Needs rays->n >= offsets[n_media] (GF_F64 rays only).
 * Errors: GF_ERR_INVALID_ARG, GF_ERR_UNSUPPORTED (GF_F32 rays), GF_ERR_CUDA.
 */
gf_status gf_trace_dopri5(gf_batch b, const gf_rays *rays, int32_t *rejects, double omega,
                          const gf_step_ctl *ctl, gf_schedule sched, const gf_tune *tune,
                          void *stream);

/*
 * gf_batch_set_precision -- evaluation mode of the batch's later
 * gf_trace_dopri5 and gf_dopri5_autotune calls: GF_F64 (default: IEEE double
 * throughout) or GF_F64X (state, stages, controller and base index law in
 * IEEE double; the Gaussian-blob sums in double-float on the FP32 pipes, as
 * gf_trace_rk4's GF_F64X).  No paper counterpart (a GB300 evaluation mode).
 * Both schedules stay bit-identical to each other in either mode.  Changing
 * the mode forgets the batch's tuned launch shape.
 * Errors: GF_ERR_INVALID_ARG (b NULL), GF_ERR_UNSUPPORTED (GF_F32).
 */
gf_status gf_batch_set_precision(gf_batch b, gf_precision prec);

/*
 * gf_dopri5_autotune -- time the persistent schedule for block size x rays per
 * thread x compaction interval x chunk on a prefix of the batch's media (about
 * an eighth of its rays, at least 65,536 when available), on scratch copies
 * of `rays` (which are not modified), and return the fastest shape in *out.
 * The result is remembered by the batch and, when cache_path is non-NULL,
 * stored in / read from that file keyed by GPU name, SM count, medium kind,
 * blob count and tolerances.  Synchronous; allocates scratch device memory.
 * Errors: as gf_trace_dopri5, plus GF_ERR_OOM.
 */
gf_status gf_dopri5_autotune(gf_batch b, const gf_rays *rays, double omega, const gf_step_ctl *ctl,
                             const char *cache_path, gf_tune *out);

#ifdef __cplusplus
}
#endif

#endif /* GF_H */
