/*
 * oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for Hamiltonian
 * ray tracing in graded-index media.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is loaded by the test-suite, by the
 * smoke check and by the CPU-baseline leg of the benchmark, nothing else.  It
 * shares no code, header, table or helper with the CUDA library; the two meet
 * only in the seeded input arrays.
 *
 * What it computes (arXiv 2508.15967, Sec. 4):
 *   - a dispersion relation D(x, k, w) that is constant along a ray (Eq. 1);
 *   - the ray equations obtained by implicit differentiation (Eqs. 2-3):
 *         dx/dt =  dw/dk = -D_k / D_w,      dk/dt = -dw/dx = D_x / D_w;
 *   - one classic 4th-order Runge-Kutta update per step, whose outputs are the
 *     updated x, k, t and the dispersion residual |D| (Sec. 4);
 *   - the initial k, chosen so that D = 0 at the launch point (Sec. 4, the
 *     initial-condition paragraph; here along a given direction, closed form);
 *   - rays that reach a cut-off (no propagating root: n^2 <= 0 or eps <= 0,
 *     equivalently D_w = 0 for w > 0) stop with a status (Sec. 4).
 * Media, adaptive Dormand-Prince stepping and the parameter sensitivities are
 * not in the paper; they follow the textbook definitions cited at each one.
 *
 * Precision: IEEE double, compiled with -ffp-contract=off (no FMA contraction),
 * no fast-math, every expression evaluated in the order written.
 *
 * Parity pins: every function here is pinned by tests that do not use this
 * file's arithmetic -- closed-form rays, invariants, central differences,
 * polynomial reproduction, order of convergence, published tableau values.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------ codes */

enum { OR_HOMOG = 0, OR_LUNEBURG = 1, OR_GRIN = 2, OR_QUADRATIC = 3, OR_SPLINE = 4, OR_COLD = 5 };

enum {
    OR_ACTIVE = 0,          /* still propagating; a further call continues it      */
    OR_EXITED = 1,          /* left the termination sphere |x| > R                  */
    OR_CUTOFF = 2,          /* reached n^2 <= 0 / eps <= 0 (D_w = 0): cut-off       */
    OR_NONFINITE = 3,       /* an update produced inf/nan; state kept before it     */
    OR_MAX_STEPS = 4,       /* adaptive stepping hit its step budget                */
    OR_STEP_UNDERFLOW = 5,  /* adaptive step fell below h_min                       */
    OR_DONE = 6             /* adaptive stepping reached t_max                      */
};

typedef struct {
    int32_t kind;
    int32_t n_blobs;
    int32_t grid_n;         /* nodes per axis of the periodic spline grid            */
    int32_t pad_;
    double n_h;             /* homogeneous index                                     */
    double n0, a;           /* GRIN: n^2 = n0^2 (1 - a^2 (y^2 + z^2))                */
    const double *blobs;    /* n_blobs rows (A, cx, cy, cz, w)                       */
    const float *grid;      /* grid_n^3 nodes x 8 floats, x fastest                  */
    int32_t n_species;      /* cold plasma: 1..4 species                             */
    int32_t pad2_;
    double species[8];      /* per species (w_p^2, Omega) at f = g = 1: squared plasma
                               frequency and signed cyclotron frequency              */
    double prof[4];         /* f(x) = prof[0] + prof[1] x_0 scales w_p^2 (density),
                               g(x) = prof[2] + prof[3] x_0 scales Omega (|B|)      */
} or_medium;

/* ------------------------------------------------------ isotropic index n^2 */

/* Squared refractive index, its gradient and (optionally) its Hessian.
 *   homogeneous : n^2 = n_h^2
 *   Luneburg    : n^2 = 2 - |x|^2 for |x|^2 <= 1, 1 outside (Luneburg 1944)
 *   quadratic   : n^2 = 2 - |x|^2 everywhere (the Luneburg law without the kink)
 *   GRIN        : n^2 = n0^2 (1 - a^2 (y^2 + z^2)) (parabolic fibre)
 * plus sum_j A_j exp(-|x - c_j|^2 / (2 w_j^2)) for every medium kind. */
static void or_index(const or_medium *m, const double *x, double *n2, double *g,
                     double H[3][3], int want_hess)
{
    int i, j, b;
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    *n2 = 0.0;
    for (i = 0; i < 3; i++) {
        g[i] = 0.0;
        if (want_hess)
            for (j = 0; j < 3; j++) H[i][j] = 0.0;
    }
    switch (m->kind) {
    case OR_HOMOG:
        *n2 = m->n_h * m->n_h;
        break;
    case OR_LUNEBURG:
        if (r2 <= 1.0) {
            *n2 = 2.0 - r2;
            for (i = 0; i < 3; i++) g[i] = -2.0 * x[i];
            if (want_hess)
                for (i = 0; i < 3; i++) H[i][i] = -2.0;
        } else {
            *n2 = 1.0;
        }
        break;
    case OR_QUADRATIC:
        *n2 = 2.0 - r2;
        for (i = 0; i < 3; i++) g[i] = -2.0 * x[i];
        if (want_hess)
            for (i = 0; i < 3; i++) H[i][i] = -2.0;
        break;
    case OR_GRIN: {
        double n02 = m->n0 * m->n0;
        double a2 = m->a * m->a;
        *n2 = n02 * (1.0 - a2 * (x[1] * x[1] + x[2] * x[2]));
        g[1] = -2.0 * n02 * a2 * x[1];
        g[2] = -2.0 * n02 * a2 * x[2];
        if (want_hess) {
            H[1][1] = -2.0 * n02 * a2;
            H[2][2] = -2.0 * n02 * a2;
        }
        break;
    }
    default:
        break;
    }
    for (b = 0; b < m->n_blobs; b++) {
        const double *bl = m->blobs + 5 * b;
        double A = bl[0], w = bl[4];
        double d[3] = { x[0] - bl[1], x[1] - bl[2], x[2] - bl[3] };
        double q = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double gb = exp(-q / (2.0 * w * w));
        *n2 += A * gb;
        for (i = 0; i < 3; i++) g[i] += A * (-gb * d[i] / (w * w));
        if (want_hess)
            for (i = 0; i < 3; i++)
                for (j = 0; j < 3; j++)
                    H[i][j] += A * gb * (d[i] * d[j] / (w * w * w * w) - (i == j ? 1.0 : 0.0) / (w * w));
    }
}

/* ------------------------------------------------ tricubic B-spline fields */

/* Uniform cubic B-spline weights of the four nodes i-1..i+2 at fraction f in
 * [0,1), and their derivatives d/df (de Boor, A Practical Guide to Splines). */
static void or_bspline(double f, double B[4], double dB[4])
{
    double u = 1.0 - f;
    B[0] = u * u * u / 6.0;
    B[1] = (3.0 * f * f * f - 6.0 * f * f + 4.0) / 6.0;
    B[2] = (-3.0 * f * f * f + 3.0 * f * f + 3.0 * f + 1.0) / 6.0;
    B[3] = f * f * f / 6.0;
    dB[0] = -u * u / 2.0;
    dB[1] = (9.0 * f * f - 12.0 * f) / 6.0;
    dB[2] = (-9.0 * f * f + 6.0 * f + 3.0) / 6.0;
    dB[3] = f * f / 2.0;
}

static int or_wrap(int64_t i, int n)
{
    int64_t r = i % n;
    return (int)(r < 0 ? r + n : r);
}

/* Values and gradients of the 7 channels (M11 M12 M13 M22 M23 M33 eps) of the
 * periodic grid on [-1,1)^3 with node spacing h = 2/n, node i at -1 + i h.
 * The stored samples are the B-spline control values (no prefilter). */
static void or_spline(const or_medium *m, const double *x, double val[7], double grad[7][3])
{
    int n = m->grid_n;
    double h = 2.0 / (double)n;
    int64_t base[3];
    double B[3][4], dB[3][4];
    int ax, a, b, c, ch;
    for (ax = 0; ax < 3; ax++) {
        double u = (x[ax] + 1.0) / h;
        double fl = floor(u);
        base[ax] = (int64_t)fl;
        or_bspline(u - fl, B[ax], dB[ax]);
        for (a = 0; a < 4; a++) dB[ax][a] = dB[ax][a] / h;
    }
    for (ch = 0; ch < 7; ch++) {
        val[ch] = 0.0;
        grad[ch][0] = grad[ch][1] = grad[ch][2] = 0.0;
    }
    for (c = 0; c < 4; c++) {
        int iz = or_wrap(base[2] - 1 + c, n);
        for (b = 0; b < 4; b++) {
            int iy = or_wrap(base[1] - 1 + b, n);
            for (a = 0; a < 4; a++) {
                int ix = or_wrap(base[0] - 1 + a, n);
                const float *node = m->grid + 8 * (((int64_t)iz * n + iy) * n + ix);
                double w = B[0][a] * B[1][b] * B[2][c];
                double wx = dB[0][a] * B[1][b] * B[2][c];
                double wy = B[0][a] * dB[1][b] * B[2][c];
                double wz = B[0][a] * B[1][b] * dB[2][c];
                for (ch = 0; ch < 7; ch++) {
                    double v = (double)node[ch];
                    val[ch] += w * v;
                    grad[ch][0] += wx * v;
                    grad[ch][1] += wy * v;
                    grad[ch][2] += wz * v;
                }
            }
        }
    }
}

/* ------------------------------------------------------ dispersion relation */

typedef struct {
    double D, Dx[3], Dk[3], Dw;
    double eps;             /* n^2 (isotropic) or eps (anisotropic): D_w = -2 w eps;
                               |D_w| for the cold plasma                            */
} or_disp;

/* Cold plasma with B along z (Sec. 4.1, Eqs. 5-10): the dielectric tensor has
 * eps11 = S = 1 - sum w_p^2 / (w^2 - Omega^2), eps12 = -i Dst with
 * Dst = sum Omega w_p^2 / (w (w^2 - Omega^2)), eps33 = P = 1 - sum w_p^2 / w^2,
 * and with n = k / w (c = 1), a = n_x^2 + n_y^2, b = n_z^2, R L = S^2 - Dst^2,
 *   D = det(eps + n n - n^2 I) = S a (a + b) + P b (a + b) - R L a - P S (a + 2 b) + P R L
 * (the Stix form A n^4 - B n^2 + C written in a and b).  The slab profiles
 * f(x) = f0 + f1 x (w_p^2 proportional to f, the linear gradient of Eq. 4)
 * and g(x) = g0 + g1 x (Omega proportional to g) depend on the first
 * coordinate only.  Gradients by the chain rule through S, Dst, P, a, b. */
static void or_cold(const or_medium *m, const double *x, const double *k, double w, or_disp *o)
{
    double f = m->prof[0] + m->prof[1] * x[0], fx = m->prof[1];
    double g = m->prof[2] + m->prof[3] * x[0], gx = m->prof[3];
    double S = 1.0, Dst = 0.0, P = 1.0, Sx = 0.0, Dx_ = 0.0, Px = 0.0, Sw = 0.0, Dw_ = 0.0, Pw = 0.0;
    double a, b, RL, DS, DD, DP, Da, Db;
    int sp;
    for (sp = 0; sp < m->n_species; sp++) {
        double wp2 = m->species[2 * sp] * f, wp2x = m->species[2 * sp] * fx;
        double W = m->species[2 * sp + 1] * g, Wx = m->species[2 * sp + 1] * gx;
        double den = w * w - W * W;
        S -= wp2 / den;
        Dst += W * wp2 / (w * den);
        P -= wp2 / (w * w);
        Sx -= (wp2x * den + 2.0 * wp2 * W * Wx) / (den * den);
        Dx_ += ((Wx * wp2 + W * wp2x) * den + 2.0 * W * W * wp2 * Wx) / (w * den * den);
        Px -= wp2x / (w * w);
        Sw += 2.0 * w * wp2 / (den * den);
        Dw_ -= W * wp2 * (3.0 * w * w - W * W) / ((w * w * w - w * W * W) * (w * w * w - w * W * W));
        Pw += 2.0 * wp2 / (w * w * w);
    }
    a = (k[0] * k[0] + k[1] * k[1]) / (w * w);
    b = k[2] * k[2] / (w * w);
    RL = S * S - Dst * Dst;
    o->D = S * a * (a + b) + P * b * (a + b) - RL * a - P * S * (a + 2.0 * b) + P * RL;
    DS = a * (a + b) - 2.0 * S * a - P * (a + 2.0 * b) + 2.0 * P * S;
    DD = 2.0 * Dst * a - 2.0 * P * Dst;
    DP = b * (a + b) - S * (a + 2.0 * b) + RL;
    Da = S * (2.0 * a + b) + P * b - RL - P * S;
    Db = S * a + P * (a + 2.0 * b) - 2.0 * P * S;
    o->Dk[0] = Da * 2.0 * k[0] / (w * w);
    o->Dk[1] = Da * 2.0 * k[1] / (w * w);
    o->Dk[2] = Db * 2.0 * k[2] / (w * w);
    o->Dx[0] = DS * Sx + DD * Dx_ + DP * Px;
    o->Dx[1] = 0.0;
    o->Dx[2] = 0.0;
    o->Dw = Da * (-2.0 * a / w) + Db * (-2.0 * b / w) + DS * Sw + DD * Dw_ + DP * Pw;
    o->eps = fabs(o->Dw);
}

/* isotropic : D = |k|^2 - w^2 n^2(x)
 * spline    : D = k^T M(x) k - w^2 eps(x)                                     */
static void or_dispersion(const or_medium *m, const double *x, const double *k, double w,
                          or_disp *o)
{
    int i, j, c;
    if (m->kind == OR_COLD) {
        or_cold(m, x, k, w, o);
        return;
    }
    if (m->kind == OR_SPLINE) {
        double val[7], grad[7][3], M[3][3], dM[3][3][3];
        static const int idx[3][3] = { { 0, 1, 2 }, { 1, 3, 4 }, { 2, 4, 5 } };
        or_spline(m, x, val, grad);
        for (i = 0; i < 3; i++)
            for (j = 0; j < 3; j++) {
                M[i][j] = val[idx[i][j]];
                for (c = 0; c < 3; c++) dM[c][i][j] = grad[idx[i][j]][c];
            }
        o->eps = val[6];
        o->D = -w * w * val[6];
        for (i = 0; i < 3; i++)
            for (j = 0; j < 3; j++) o->D += k[i] * M[i][j] * k[j];
        for (i = 0; i < 3; i++) {
            o->Dk[i] = 0.0;
            for (j = 0; j < 3; j++) o->Dk[i] += 2.0 * M[i][j] * k[j];
        }
        for (c = 0; c < 3; c++) {
            o->Dx[c] = -w * w * grad[6][c];
            for (i = 0; i < 3; i++)
                for (j = 0; j < 3; j++) o->Dx[c] += k[i] * dM[c][i][j] * k[j];
        }
        o->Dw = -2.0 * w * val[6];
    } else {
        double n2, g[3], H[3][3];
        or_index(m, x, &n2, g, H, 0);
        o->eps = n2;
        o->D = k[0] * k[0] + k[1] * k[1] + k[2] * k[2] - w * w * n2;
        for (i = 0; i < 3; i++) {
            o->Dk[i] = 2.0 * k[i];
            o->Dx[i] = -w * w * g[i];
        }
        o->Dw = -2.0 * w * n2;
    }
}

/* Ray right-hand side, Eqs. 2-3: f = (-D_k / D_w, D_x / D_w).
 * Returns OR_CUTOFF where the medium has no propagating root (eps <= 0). */
static int or_rhs(const or_medium *m, const double *y, double w, double *f, double *D)
{
    or_disp d;
    int i;
    or_dispersion(m, y, y + 3, w, &d);
    if (D) *D = d.D;
    if (!(d.eps > 0.0)) return OR_CUTOFF;
    for (i = 0; i < 3; i++) {
        f[i] = -d.Dk[i] / d.Dw;
        f[3 + i] = d.Dx[i] / d.Dw;
    }
    return OR_ACTIVE;
}

static double fmax_d(double a, double b) { return a > b ? a : b; }
static double fmin_d(double a, double b) { return a < b ? a : b; }

static int or_finite6(const double *y)
{
    int i;
    for (i = 0; i < 6; i++)
        if (!isfinite(y[i])) return 0;
    return 1;
}

/* ------------------------------------------------------------ public: eval */

/* D and its partials at n points (x, k given as (n,3) row-major arrays).
 * out: (n, 9) rows (D, Dx0, Dx1, Dx2, Dk0, Dk1, Dk2, Dw, eps). */
void or_eval(const or_medium *m, int64_t n, const double *x, const double *k, double w,
             double *out)
{
    int64_t r;
#pragma omp parallel for schedule(static)
    for (r = 0; r < n; r++) {
        or_disp d;
        int i;
        or_dispersion(m, x + 3 * r, k + 3 * r, w, &d);
        out[9 * r] = d.D;
        for (i = 0; i < 3; i++) {
            out[9 * r + 1 + i] = d.Dx[i];
            out[9 * r + 4 + i] = d.Dk[i];
        }
        out[9 * r + 7] = d.Dw;
        out[9 * r + 8] = d.eps;
    }
}

/* n^2, grad n^2 and Hessian of n^2 at n points: out (n, 13) = (n2, g[3], H[9]). */
void or_index_hess(const or_medium *m, int64_t n, const double *x, double *out)
{
    int64_t r;
    for (r = 0; r < n; r++) {
        double n2, g[3], H[3][3];
        int i, j;
        or_index(m, x + 3 * r, &n2, g, H, 1);
        out[13 * r] = n2;
        for (i = 0; i < 3; i++) out[13 * r + 1 + i] = g[i];
        for (i = 0; i < 3; i++)
            for (j = 0; j < 3; j++) out[13 * r + 4 + 3 * i + j] = H[i][j];
    }
}

/* --------------------------------------------------------- public: on-shell */

/* k0 = s d with s > 0 chosen so that D(x0, s d, w) = 0.  Both media are
 * quadratic in k along a fixed direction, D(s d) = s^2 q - w^2 eps, so
 * s = w sqrt(eps / q) with q = d.d (isotropic) or d^T M d (spline).
 * status[r] = OR_CUTOFF (k0 = 0) where eps <= 0. */
void or_onshell(const or_medium *m, int64_t n, const double *x0, const double *dir, double w,
                double *k0, int32_t *status)
{
    int64_t r;
#pragma omp parallel for schedule(static)
    for (r = 0; r < n; r++) {
        const double *x = x0 + 3 * r, *d = dir + 3 * r;
        double eps, q, s;
        int i, j;
        if (m->kind == OR_COLD) {     /* two branches: use or_newton_kx instead */
            status[r] = OR_CUTOFF;
            for (i = 0; i < 3; i++) k0[3 * r + i] = 0.0;
            continue;
        }
        if (m->kind == OR_SPLINE) {
            double val[7], grad[7][3];
            static const int idx[3][3] = { { 0, 1, 2 }, { 1, 3, 4 }, { 2, 4, 5 } };
            or_spline(m, x, val, grad);
            eps = val[6];
            q = 0.0;
            for (i = 0; i < 3; i++)
                for (j = 0; j < 3; j++) q += d[i] * val[idx[i][j]] * d[j];
        } else {
            double g[3], H[3][3];
            or_index(m, x, &eps, g, H, 0);
            q = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        }
        if (!(eps > 0.0) || !(q > 0.0)) {
            status[r] = OR_CUTOFF;
            for (i = 0; i < 3; i++) k0[3 * r + i] = 0.0;
            continue;
        }
        s = w * sqrt(eps / q);
        status[r] = OR_ACTIVE;
        for (i = 0; i < 3; i++) k0[3 * r + i] = s * d[i];
    }
}

/* ------------------------------------------------------ public: Newton k_x */

/* The paper's ray initialisation (Sec. 4): w, x, k_y and k_z are fixed and
 * k_x solves D(x, k, w) = 0 by Newton's method, k_x <- k_x - D / (dD/dk_x),
 * to |D| < tol; the initial guess (k_x on entry) selects the root.  An
 * iteration also stops, converged, when its step no longer changes k_x beyond
 * rounding (|dk_x| <= 2^-50 |k_x|) with |D| <= 8 tol.  Rays that do not
 * converge in max_iter steps, or meet dD/dk_x = 0, get OR_CUTOFF (no
 * propagating root) and keep their last k_x.  k: (n, 3) in/out; iters: (n,). */
void or_newton_kx(const or_medium *m, int64_t n, const double *x, double *k, double w, double tol,
                  int max_iter, int32_t *status, int32_t *iters)
{
    int64_t r;
#pragma omp parallel for schedule(static)
    for (r = 0; r < n; r++) {
        double *kr = k + 3 * r;
        int it, ok = 0;
        for (it = 0; it < max_iter; it++) {
            or_disp d;
            double step;
            or_dispersion(m, x + 3 * r, kr, w, &d);
            if (fabs(d.D) < tol) { ok = 1; break; }
            if (d.Dk[0] == 0.0 || !isfinite(d.D)) break;
            step = d.D / d.Dk[0];
            kr[0] = kr[0] - step;
            if (fabs(step) <= 0x1p-50 * fabs(kr[0])) {
                or_dispersion(m, x + 3 * r, kr, w, &d);
                ok = fabs(d.D) <= 8.0 * tol;
                it++;
                break;
            }
        }
        status[r] = ok ? OR_ACTIVE : OR_CUTOFF;
        iters[r] = it;
    }
}

/* ------------------------------------------------------------ public: RK4 */

/* One ray, classic RK4 with fixed dt for up to n_steps steps (Sec. 4):
 *   K1 = f(y), K2 = f(y + dt/2 K1), K3 = f(y + dt/2 K2), K4 = f(y + dt K3),
 *   y <- y + dt/6 (K1 + 2 K2 + 2 K3 + K4),   t_n = t_0 + n dt.
 * Residual bookkeeping: dmax <- max(dmax, |D(y_n)|) over every state visited
 * (the stage-1 evaluation of each step and the final state); dres = |D(final)|.
 * ckpt (may be NULL): state before step j*every stored at ckpt[j*6 .. j*6+5]. */
static double or_kink(const double *Y)
{
    return fabs(Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2] - 1.0);
}

/* kink (may be NULL): min over every stage point of ||x|^2 - 1|, the distance
 * in |x|^2 from the Luneburg surface where grad n^2 jumps. */
static void or_rk4_ray(const or_medium *m, double *y, double *t, int32_t *status, int32_t *steps,
                       double *dres, double *dmax, double w, double dt, int64_t n_steps,
                       double radius, int64_t every, double *ckpt, double *kink)
{
    double K1[6], K2[6], K3[6], K4[6], Y[6], yn[6], D;
    double t0 = *t, dm = *dmax;
    int64_t s;
    int i, st;
    if (*status != OR_ACTIVE) return;
    for (s = 0; s < n_steps; s++) {
        if (ckpt && every > 0 && s % every == 0)
            for (i = 0; i < 6; i++) ckpt[6 * (s / every) + i] = y[i];
        st = or_rhs(m, y, w, K1, &D);
        if (kink && or_kink(y) < *kink) *kink = or_kink(y);
        if (fabs(D) > dm) dm = fabs(D);
        if (st != OR_ACTIVE) { *status = st; break; }
        for (i = 0; i < 6; i++) Y[i] = y[i] + (dt / 2.0) * K1[i];
        if (kink && or_kink(Y) < *kink) *kink = or_kink(Y);
        st = or_rhs(m, Y, w, K2, NULL);
        if (st != OR_ACTIVE) { *status = st; break; }
        for (i = 0; i < 6; i++) Y[i] = y[i] + (dt / 2.0) * K2[i];
        if (kink && or_kink(Y) < *kink) *kink = or_kink(Y);
        st = or_rhs(m, Y, w, K3, NULL);
        if (st != OR_ACTIVE) { *status = st; break; }
        for (i = 0; i < 6; i++) Y[i] = y[i] + dt * K3[i];
        if (kink && or_kink(Y) < *kink) *kink = or_kink(Y);
        st = or_rhs(m, Y, w, K4, NULL);
        if (st != OR_ACTIVE) { *status = st; break; }
        for (i = 0; i < 6; i++)
            yn[i] = y[i] + (dt / 6.0) * (K1[i] + 2.0 * K2[i] + 2.0 * K3[i] + K4[i]);
        if (!or_finite6(yn)) { *status = OR_NONFINITE; break; }
        for (i = 0; i < 6; i++) y[i] = yn[i];
        *steps += 1;
        *t = t0 + (double)(s + 1) * dt;
        if (radius > 0.0 && y[0] * y[0] + y[1] * y[1] + y[2] * y[2] > radius * radius) {
            *status = OR_EXITED;
            break;
        }
    }
    {
        or_disp d;
        or_dispersion(m, y, y + 3, w, &d);
        if (fabs(d.D) > dm) dm = fabs(d.D);
        *dres = fabs(d.D);
        *dmax = dm;
    }
}

/* y: (n, 6) rows (x, y, z, kx, ky, kz); t, status, steps, dres, dmax: (n,).
 * ckpt (may be NULL): (n, n_ckpt, 6), n_ckpt = ceil(n_steps / every). */
void or_trace_rk4(const or_medium *m, int64_t n, double *y, double *t, int32_t *status,
                  int32_t *steps, double *dres, double *dmax, double w, double dt,
                  int64_t n_steps, double radius, int64_t every, double *ckpt)
{
    int64_t r, nck = (every > 0) ? (n_steps + every - 1) / every : 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (r = 0; r < n; r++)
        or_rk4_ray(m, y + 6 * r, t + r, status + r, steps + r, dres + r, dmax + r, w, dt,
                   n_steps, radius, every, ckpt ? ckpt + 6 * nck * r : NULL, NULL);
}

/* As or_trace_rk4 without checkpoints, also returning kink[r] (initialise to a
 * large value): the minimum over all stage points of ||x|^2 - 1|. */
void or_trace_rk4_kink(const or_medium *m, int64_t n, double *y, double *t, int32_t *status,
                       int32_t *steps, double *dres, double *dmax, double w, double dt,
                       int64_t n_steps, double radius, double *kink)
{
    int64_t r;
#pragma omp parallel for schedule(dynamic, 16)
    for (r = 0; r < n; r++)
        or_rk4_ray(m, y + 6 * r, t + r, status + r, steps + r, dres + r, dmax + r, w, dt,
                   n_steps, radius, 0, NULL, kink + r);
}

/* -------------------------------------------------------- public: DOPRI5 */

/* Dormand-Prince 5(4) tableau: J. R. Dormand and P. J. Prince, "A family of
 * embedded Runge-Kutta formulae", J. Comput. Appl. Math. 6 (1980) 19-26;
 * tabulated in Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.5. */
static const double DP_C[7] = { 0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0 };
static const double DP_A[7][6] = {
    { 0, 0, 0, 0, 0, 0 },
    { 1.0 / 5.0, 0, 0, 0, 0, 0 },
    { 3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0 },
    { 44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0 },
    { 19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0 },
    { 9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0 },
    { 35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0 },
};
/* 5th-order weights (= last row of A, first-same-as-last) and 4th-order weights */
static const double DP_B[7] = { 35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0,
                                -2187.0 / 6784.0, 11.0 / 84.0, 0.0 };
static const double DP_BS[7] = { 5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                                 -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0 };

/* Tableau export for the tests: out[0..6]=c, [7..48]=A (7x6), [49..55]=b, [56..62]=b*. */
void or_dopri5_tableau(double *out)
{
    int i, j;
    for (i = 0; i < 7; i++) out[i] = DP_C[i];
    for (i = 0; i < 7; i++)
        for (j = 0; j < 6; j++) out[7 + 6 * i + j] = DP_A[i][j];
    for (i = 0; i < 7; i++) out[49 + i] = DP_B[i];
    for (i = 0; i < 7; i++) out[56 + i] = DP_BS[i];
}

typedef struct {
    double rtol, atol, h0, t_max, radius;
    double fac_min, fac_max, safety;
    int64_t max_steps;
} or_step_ctl;

/* One ray, adaptive DOPRI5 with the step-size controller of Hairer-Norsett-
 * Wanner I, Sec. II.4: err = sqrt(mean_i (e_i / sc_i)^2) with
 * sc_i = atol + rtol max(|y_i|, |y_new,i|); accept iff err <= 1;
 * h <- h min(fac_max, max(fac_min, safety err^(-1/5))), growth capped at 1 on
 * the step after a rejection; the last step is shortened to land on t_max.
 * Terminates: EXITED after an accepted step ending outside |x| = radius (no
 * event location), DONE at t_max, MAX_STEPS after max_steps accepted steps,
 * STEP_UNDERFLOW when h < 1e-14 max(1, |t|), CUTOFF / NONFINITE as in RK4. */
static void or_dopri5_ray(const or_medium *m, const or_step_ctl *c, double w, double *y,
                          double *t, int32_t *status, int32_t *steps, int32_t *rejects,
                          double *dres, double *dmax)
{
    double K[7][6], Y[6], yn[6], h = c->h0, D, dm = *dmax, fmax = c->fac_max;
    int i, j, st;
    if (*status != OR_ACTIVE) return;
    st = or_rhs(m, y, w, K[0], &D);
    if (fabs(D) > dm) dm = fabs(D);
    if (st != OR_ACTIVE) *status = st;
    while (*status == OR_ACTIVE) {
        double err, fac, hs;
        int last = 0, bad = 0;
        if (*steps >= c->max_steps) { *status = OR_MAX_STEPS; break; }
        if (*t >= c->t_max) { *status = OR_DONE; break; }
        hs = h;
        if (*t + hs >= c->t_max) { hs = c->t_max - *t; last = 1; }
        if (hs < 1e-14 * fmax_d(1.0, fabs(*t))) { *status = OR_STEP_UNDERFLOW; break; }
        for (j = 1; j < 7 && !bad; j++) {
            for (i = 0; i < 6; i++) {
                double acc = 0.0;
                int l;
                for (l = 0; l < j; l++) acc += DP_A[j][l] * K[l][i];
                Y[i] = y[i] + hs * acc;
            }
            st = or_rhs(m, Y, w, K[j], j == 6 ? &D : NULL);
            if (st != OR_ACTIVE) { *status = st; bad = 1; }
        }
        if (bad) break;
        /* the stage-7 point is the 5th-order solution (b = last row of A) */
        for (i = 0; i < 6; i++) yn[i] = Y[i];
        if (!or_finite6(yn) || !or_finite6(K[6])) { *status = OR_NONFINITE; break; }
        err = 0.0;
        for (i = 0; i < 6; i++) {
            double e = 0.0, sc;
            int l;
            for (l = 0; l < 7; l++) e += (DP_B[l] - DP_BS[l]) * K[l][i];
            e = hs * e;
            sc = c->atol + c->rtol * fmax_d(fabs(y[i]), fabs(yn[i]));
            err += (e / sc) * (e / sc);
        }
        err = sqrt(err / 6.0);
        fac = (err > 0.0) ? c->safety * pow(err, -0.2) : fmax;
        if (err <= 1.0) {
            for (i = 0; i < 6; i++) { y[i] = yn[i]; K[0][i] = K[6][i]; }
            *t = last ? c->t_max : *t + hs;
            *steps += 1;
            if (fabs(D) > dm) dm = fabs(D);
            h = hs * fmin_d(fmax, fmax_d(c->fac_min, fac));
            fmax = c->fac_max;
            if (c->radius > 0.0 && y[0] * y[0] + y[1] * y[1] + y[2] * y[2] > c->radius * c->radius)
                *status = OR_EXITED;
        } else {
            *rejects += 1;
            h = hs * fmin_d(fmax, fmax_d(c->fac_min, fac));
            fmax = 1.0;
        }
    }
    {
        or_disp d;
        or_dispersion(m, y, y + 3, w, &d);
        if (fabs(d.D) > dm) dm = fabs(d.D);
        *dres = fabs(d.D);
        *dmax = dm;
    }
}

/* Many media, rays of medium j in [offsets[j], offsets[j+1]); same layouts as
 * or_trace_rk4.  media: n_media descriptions. */
void or_trace_dopri5(const or_medium *media, int64_t n_media, const int64_t *offsets,
                     double *y, double *t, int32_t *status, int32_t *steps, int32_t *rejects,
                     double *dres, double *dmax, double w, const or_step_ctl *c)
{
    int64_t j;
    for (j = 0; j < n_media; j++) {
        int64_t r, lo = offsets[j], hi = offsets[j + 1];
#pragma omp parallel for schedule(dynamic, 4)
        for (r = lo; r < hi; r++)
            or_dopri5_ray(media + j, c, w, y + 6 * r, t + r, status + r, steps + r, rejects + r,
                          dres + r, dmax + r);
    }
}

/* ---------------------------------------------- public: tangent-linear RK4 */

/* Jacobian of the ray right-hand side and its derivative with respect to the
 * blob amplitudes, for isotropic media, written from f = (-D_k/D_w, D_x/D_w)
 * by the quotient rule with the second derivatives of D = |k|^2 - w^2 n^2:
 *   D_kk = 2 I, D_kx = 0, D_xx = -w^2 Hess(n^2), dD_w/dx = -2 w grad(n^2),
 *   dD/dA_j = -w^2 g_j, dD_x/dA_j = -w^2 grad g_j, dD_w/dA_j = -2 w g_j.
 * J: 6x6 row-major (d f_r / d y_c); Ft: 6 x nb (d f_r / d A_j). */
static int or_rhs_jac(const or_medium *m, const double *y, double w, double *f, double J[6][6],
                      double *Ft)
{
    double n2, g[3], H[3][3], Dw, Dk[3], Dx[3], dDw_dx[3];
    int i, j, b, nb = m->n_blobs;
    const double *x = y, *k = y + 3;
    or_index(m, x, &n2, g, H, 1);
    if (!(n2 > 0.0)) return OR_CUTOFF;
    Dw = -2.0 * w * n2;
    for (i = 0; i < 3; i++) {
        Dk[i] = 2.0 * k[i];
        Dx[i] = -w * w * g[i];
        dDw_dx[i] = -2.0 * w * g[i];
    }
    for (i = 0; i < 3; i++) {
        f[i] = -Dk[i] / Dw;
        f[3 + i] = Dx[i] / Dw;
    }
    for (i = 0; i < 6; i++)
        for (j = 0; j < 6; j++) J[i][j] = 0.0;
    for (i = 0; i < 3; i++) {
        for (j = 0; j < 3; j++) {
            /* d(-D_k_i / D_w)/dx_j = -D_kx_ij / D_w + D_k_i dD_w/dx_j / D_w^2, D_kx = 0 */
            J[i][j] = Dk[i] * dDw_dx[j] / (Dw * Dw);
            /* d(-D_k_i / D_w)/dk_j = -D_kk_ij / D_w, dD_w/dk = 0 */
            J[i][3 + j] = -(i == j ? 2.0 : 0.0) / Dw;
            /* d(D_x_i / D_w)/dx_j = D_xx_ij / D_w - D_x_i dD_w/dx_j / D_w^2 */
            J[3 + i][j] = (-w * w * H[i][j]) / Dw - Dx[i] * dDw_dx[j] / (Dw * Dw);
            /* d(D_x_i / D_w)/dk_j = 0 */
        }
    }
    for (b = 0; b < nb; b++) {
        const double *bl = m->blobs + 5 * b;
        double wb = bl[4];
        double d[3] = { x[0] - bl[1], x[1] - bl[2], x[2] - bl[3] };
        double q = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double gb = exp(-q / (2.0 * wb * wb));
        double dDw = -2.0 * w * gb;
        for (i = 0; i < 3; i++) {
            double dgrad = -gb * d[i] / (wb * wb);
            double dDx = -w * w * dgrad;
            Ft[i * nb + b] = Dk[i] * dDw / (Dw * Dw);
            Ft[(3 + i) * nb + b] = dDx / Dw - Dx[i] * dDw / (Dw * Dw);
        }
    }
    return OR_ACTIVE;
}

/* Forward (tangent-linear) sensitivities S = dy/dA of the RK4 map, for
 * isotropic media, propagated alongside the trajectory: with Ydot_1 = S,
 * Ydot_i = S + a_i dt Kdot_{i-1}, Kdot_i = J(Y_i) Ydot_i + F_A(Y_i),
 * S <- S + dt/6 (Kdot_1 + 2 Kdot_2 + 2 Kdot_3 + Kdot_4).
 * Same stopping rules as or_trace_rk4 (a stopped ray keeps its S).
 * S: (n, 6, nb), zero on entry for a trace from the launch state. */
void or_tangent_rk4(const or_medium *m, int64_t n, double *y, double *t, int32_t *status,
                    int32_t *steps, double *S, double w, double dt, int64_t n_steps, double radius)
{
    int64_t r;
    int nb = m->n_blobs;
#pragma omp parallel for schedule(dynamic, 4)
    for (r = 0; r < n; r++) {
        double *yr = y + 6 * r, *Sr = S + (int64_t)6 * nb * r;
        double K[4][6], Y[6], J[6][6], yn[6];
        double *Kd = (double *)__builtin_alloca(sizeof(double) * 4 * 6 * nb);
        double *Yd = (double *)__builtin_alloca(sizeof(double) * 6 * nb);
        double *Ft = (double *)__builtin_alloca(sizeof(double) * 6 * nb);
        static const double a[4] = { 0.0, 0.5, 0.5, 1.0 };
        double t0 = t[r];
        int64_t s;
        int i, j, b, st, stage;
        if (status[r] != OR_ACTIVE) continue;
        for (s = 0; s < n_steps; s++) {
            st = OR_ACTIVE;
            for (stage = 0; stage < 4 && st == OR_ACTIVE; stage++) {
                for (i = 0; i < 6; i++) {
                    Y[i] = (stage == 0) ? yr[i] : yr[i] + (a[stage] * dt) * K[stage - 1][i];
                    for (b = 0; b < nb; b++)
                        Yd[i * nb + b] = (stage == 0) ? Sr[i * nb + b]
                            : Sr[i * nb + b] + (a[stage] * dt) * Kd[(stage - 1) * 6 * nb + i * nb + b];
                }
                st = or_rhs_jac(m, Y, w, K[stage], J, Ft);
                if (st != OR_ACTIVE) break;
                for (i = 0; i < 6; i++)
                    for (b = 0; b < nb; b++) {
                        double acc = Ft[i * nb + b];
                        for (j = 0; j < 6; j++) acc += J[i][j] * Yd[j * nb + b];
                        Kd[stage * 6 * nb + i * nb + b] = acc;
                    }
            }
            if (st != OR_ACTIVE) { status[r] = st; break; }
            for (i = 0; i < 6; i++)
                yn[i] = yr[i] + (dt / 6.0) * (K[0][i] + 2.0 * K[1][i] + 2.0 * K[2][i] + K[3][i]);
            if (!or_finite6(yn)) { status[r] = OR_NONFINITE; break; }
            for (i = 0; i < 6; i++) {
                yr[i] = yn[i];
                for (b = 0; b < nb; b++)
                    Sr[i * nb + b] = Sr[i * nb + b] + (dt / 6.0) *
                        (Kd[0 * 6 * nb + i * nb + b] + 2.0 * Kd[1 * 6 * nb + i * nb + b] +
                         2.0 * Kd[2 * 6 * nb + i * nb + b] + Kd[3 * 6 * nb + i * nb + b]);
            }
            steps[r] += 1;
            t[r] = t0 + (double)(s + 1) * dt;
            if (radius > 0.0 && yr[0] * yr[0] + yr[1] * yr[1] + yr[2] * yr[2] > radius * radius) {
                status[r] = OR_EXITED;
                break;
            }
        }
    }
}

/* dL/dA for L = sum_r |x_N,r - x*_r|^2 from the sensitivities: (nb,) output. */
void or_loss_grad(int64_t n, int nb, const double *y, const double *xstar, const double *S,
                  double *grad)
{
    int64_t r;
    int b, i;
    for (b = 0; b < nb; b++) grad[b] = 0.0;
    for (r = 0; r < n; r++)
        for (i = 0; i < 3; i++) {
            double e = 2.0 * (y[6 * r + i] - xstar[3 * r + i]);
            for (b = 0; b < nb; b++) grad[b] += e * S[(int64_t)6 * nb * r + i * nb + b];
        }
}

/* Threads OpenMP would use, for the benchmark's core count. */
int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
