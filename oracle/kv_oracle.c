/*
 * kv_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the reduced
 * Kelvin-Voigt shear-wave method.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or call
 * this file; only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark do. It shares no code with the CUDA library.
 *
 * Every routine is written from the paper's definitions, in its order:
 *   - Sec. 3.1  explicit FDTD update (3-level leapfrog, acceleration a^n with
 *               mu/rho Laplacian, eta/rho Laplacian of the backward velocity,
 *               f_S/rho), 7-point Laplacian, Dirichlet outer layer (Sec. 3.5).
 *   - Sec. 3.2  solenoidal projection: grad phi + f_S = f, Poisson equation for
 *               phi, masked matrix-free CG with the paper's recurrences and
 *               stopping rule and guards.
 *   - Sec. 3.3  pre-computed projection for separable forces: f_S^n = g(t_n) f_S0.
 *
 * Grid: nx*ny*nz nodes, x fastest, idx = (k*ny + j)*nx + i, spacing dx on all
 * axes. The outer node layer is the Dirichlet layer; the interior mask m is 1
 * for 1 <= i <= nx-2 (and likewise in y, z) and 0 elsewhere.
 *
 * Readings of points the paper leaves open (each listed in the design notes):
 *   - collocated nodes for all three displacement components;
 *   - discrete divergence = backward differences D-, discrete gradient =
 *     forward differences D+, so that D-(D+ phi) is the 7-point Laplacian;
 *   - Poisson right-hand side b = -(D- . f) on interior nodes (the divergence
 *     reads the force on the outer layer too), so that A phi = b with A = -L
 *     solves L phi = div f, and f_S = f - D+ phi on every node (Sec. 3.2.1);
 *     then D- . f_S = -(b - A phi) exactly and the projection is idempotent;
 *   - the CG stops on the paper's relative residual; the true residual
 *     ||b - A phi|| / ||b|| is reported alongside.
 *
 * Elementwise loops may run under OpenMP (the arithmetic of each output value
 * is unchanged); every reduction is a plain serial loop in index order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, k) ((((size_t)(k)) * (size_t)ny + (size_t)(j)) * (size_t)nx + (size_t)(i))

static int g_threads = 1;

void or_set_threads(int n)
{
    g_threads = n < 1 ? 1 : n;
#ifdef _OPENMP
    omp_set_num_threads(g_threads);
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return g_threads;
#else
    return 1;
#endif
}

static int is_interior(int i, int j, int k, int nx, int ny, int nz)
{
    return i > 0 && i < nx - 1 && j > 0 && j < ny - 1 && k > 0 && k < nz - 1;
}

/* Sec. 3.1: 7-point second-order Laplacian on interior nodes,
 * (L q)_ijk = sum over axes (q_{+1} - 2 q + q_{-1}) / dx^2. Boundary output = 0. */
void or_laplacian(int nx, int ny, int nz, double dx, const double *q, double *out)
{
    const double inv = 1.0 / (dx * dx);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(i, j, k);
                if (!is_interior(i, j, k, nx, ny, nz)) {
                    out[c] = 0.0;
                    continue;
                }
                double sx = q[IDX(i + 1, j, k)] - 2.0 * q[c] + q[IDX(i - 1, j, k)];
                double sy = q[IDX(i, j + 1, k)] - 2.0 * q[c] + q[IDX(i, j - 1, k)];
                double sz = q[IDX(i, j, k + 1)] - 2.0 * q[c] + q[IDX(i, j, k - 1)];
                out[c] = (sx + sy + sz) * inv;
            }
}

/* A q = -(L q) restricted to the interior (Sec. 3.2.3: A = -nabla_h^2). */
void or_apply_A(int nx, int ny, int nz, double dx, const double *q, double *out)
{
    size_t N = (size_t)nx * ny * nz;
    or_laplacian(nx, ny, nz, dx, q, out);
    #pragma omp parallel for schedule(static)
    for (size_t c = 0; c < N; ++c) out[c] = -out[c];
}

/* Discrete divergence with backward differences on interior nodes,
 * (D- . f)_ijk = (fx_ijk - fx_{i-1}) + (fy_ijk - fy_{j-1}) + (fz_ijk - fz_{k-1}), / dx.
 * Boundary output = 0. */
void or_div_minus(int nx, int ny, int nz, double dx, const double *fx, const double *fy,
                  const double *fz, double *out)
{
    const double inv = 1.0 / dx;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(i, j, k);
                if (!is_interior(i, j, k, nx, ny, nz)) {
                    out[c] = 0.0;
                    continue;
                }
                double d = (fx[c] - fx[IDX(i - 1, j, k)]) + (fy[c] - fy[IDX(i, j - 1, k)]) +
                           (fz[c] - fz[IDX(i, j, k - 1)]);
                out[c] = d * inv;
            }
}

/* Discrete gradient with forward differences at every node,
 * (D+ phi)_x = (phi_{i+1} - phi_i)/dx, with phi = 0 beyond the last node. */
void or_grad_plus(int nx, int ny, int nz, double dx, const double *phi, double *gx, double *gy,
                  double *gz)
{
    const double inv = 1.0 / dx;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(i, j, k);
                double p = phi[c];
                double px = (i + 1 < nx) ? phi[IDX(i + 1, j, k)] : 0.0;
                double py = (j + 1 < ny) ? phi[IDX(i, j + 1, k)] : 0.0;
                double pz = (k + 1 < nz) ? phi[IDX(i, j, k + 1)] : 0.0;
                gx[c] = (px - p) * inv;
                gy[c] = (py - p) * inv;
                gz[c] = (pz - p) * inv;
            }
}

static void apply_mask(int nx, int ny, int nz, double *q)
{
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                if (!is_interior(i, j, k, nx, ny, nz)) q[IDX(i, j, k)] = 0.0;
}

static double dot(size_t N, const double *a, const double *b)
{
    double s = 0.0;
    for (size_t c = 0; c < N; ++c) s += a[c] * b[c];
    return s;
}

/* Status codes of the oracle's CG (Sec. 3.2.3 stopping rule and guards). */
enum { OR_CG_CONVERGED = 0, OR_CG_MAXITER = 1, OR_CG_BREAKDOWN = 2, OR_CG_NONFINITE = 3,
       OR_CG_ZERO_RHS = 4 };

/*
 * Sec. 3.2.3: masked matrix-free CG for A phi = b, A = -L on interior nodes.
 *   r0 = (b - A phi0) m, p0 = r0
 *   alpha_k = r_k.r_k / p_k.A p_k
 *   phi_{k+1} = (phi_k + alpha_k p_k) m
 *   r_{k+1}   = (r_k - alpha_k A p_k) m
 *   beta_k    = r_{k+1}.r_{k+1} / r_k.r_k
 *   p_{k+1}   = (r_{k+1} + beta_k p_k) m
 * Stops when sqrt(|r_k|^2 / |r_0|^2) < tol, after max_iter iterations, or when
 * the denominator p.Ap or the residual becomes non-finite or non-positive.
 * phi holds phi0 on entry (zeros for the paper's start) and the result on exit.
 * out_stats[0] = iterations, [1] = final recursive relative residual,
 * [2] = true relative residual ||b - A phi|| / ||b||.
 */
int or_cg(int nx, int ny, int nz, double dx, const double *b, double *phi, double tol,
          int max_iter, double *out_stats)
{
    size_t N = (size_t)nx * ny * nz;
    double *r = (double *)malloc(N * sizeof(double));
    double *p = (double *)malloc(N * sizeof(double));
    double *Ap = (double *)malloc(N * sizeof(double));
    int status = OR_CG_MAXITER, it = 0;
    double rel = 0.0;

    apply_mask(nx, ny, nz, phi);
    or_apply_A(nx, ny, nz, dx, phi, Ap);
    #pragma omp parallel for schedule(static)
    for (size_t c = 0; c < N; ++c) r[c] = b[c] - Ap[c];
    apply_mask(nx, ny, nz, r);
    memcpy(p, r, N * sizeof(double));
    double rr = dot(N, r, r);
    const double rr0 = rr;
    if (!isfinite(rr0)) {
        status = OR_CG_NONFINITE;
        goto done;
    }
    if (rr0 == 0.0) {
        status = OR_CG_ZERO_RHS;
        goto done;
    }
    rel = 1.0;
    for (it = 0; it < max_iter;) {
        or_apply_A(nx, ny, nz, dx, p, Ap);
        double pAp = dot(N, p, Ap);
        if (!isfinite(pAp) || pAp <= 0.0) {
            status = OR_CG_BREAKDOWN;
            break;
        }
        double alpha = rr / pAp;
        #pragma omp parallel for schedule(static)
        for (size_t c = 0; c < N; ++c) phi[c] = phi[c] + alpha * p[c];
        apply_mask(nx, ny, nz, phi);
        #pragma omp parallel for schedule(static)
        for (size_t c = 0; c < N; ++c) r[c] = r[c] - alpha * Ap[c];
        apply_mask(nx, ny, nz, r);
        double rr_new = dot(N, r, r);
        ++it;
        if (!isfinite(rr_new)) {
            status = OR_CG_NONFINITE;
            break;
        }
        rel = sqrt(rr_new / rr0);
        if (rel < tol) {
            status = OR_CG_CONVERGED;
            break;
        }
        if (rr_new <= 0.0) {
            status = OR_CG_BREAKDOWN;
            break;
        }
        double beta = rr_new / rr;
        #pragma omp parallel for schedule(static)
        for (size_t c = 0; c < N; ++c) p[c] = r[c] + beta * p[c];
        apply_mask(nx, ny, nz, p);
        rr = rr_new;
    }
done:
    if (out_stats) {
        double bb = dot(N, b, b);
        or_apply_A(nx, ny, nz, dx, phi, Ap);
        #pragma omp parallel for schedule(static)
        for (size_t c = 0; c < N; ++c) r[c] = b[c] - Ap[c];
        apply_mask(nx, ny, nz, r);
        out_stats[0] = (double)it;
        out_stats[1] = rel;
        out_stats[2] = bb > 0.0 ? sqrt(dot(N, r, r) / bb) : 0.0;
    }
    free(r);
    free(p);
    free(Ap);
    return status;
}

/*
 * Sec. 3.2.1 / 3.3: solenoidal projection of a force pattern f.
 *   b   = -(D- . f) on interior nodes   (A phi = b  <=>  L phi = div f)
 *   CG  : A phi = b from phi = 0
 *   f_S = f - D+ phi on every node      (the step only reads interior ones)
 * Outputs phi (N) and fs (3N, component-major); out_stats as in or_cg.
 */
int or_project(int nx, int ny, int nz, double dx, const double *f /*3N*/, double tol,
               int max_iter, double *phi, double *fs /*3N*/, double *out_stats)
{
    size_t N = (size_t)nx * ny * nz;
    double *b = (double *)malloc(N * sizeof(double));
    or_div_minus(nx, ny, nz, dx, f, f + N, f + 2 * N, b);
    #pragma omp parallel for schedule(static)
    for (size_t c = 0; c < N; ++c) b[c] = -b[c];
    memset(phi, 0, N * sizeof(double));
    int st = or_cg(nx, ny, nz, dx, b, phi, tol, max_iter, out_stats);
    or_grad_plus(nx, ny, nz, dx, phi, fs, fs + N, fs + 2 * N);
    #pragma omp parallel for schedule(static)
    for (size_t c = 0; c < 3 * N; ++c) fs[c] = f[c] - fs[c];
    free(b);
    return st;
}

/*
 * Sec. 3.1 / 3.3: explicit leapfrog time stepping with the pre-computed
 * projection, written as the 3-level recurrence
 *   u^{n+1} = 2 u^n - u^{n-1} + dt^2 a^n,
 *   a^n = (mu/rho) L u^n + (eta/rho) L udot^n + (g_n/rho) f_S0,
 *   udot^n = (u^n - u^{n-1}) / dt,
 * on interior nodes; u = 0 on the outer layer (Sec. 3.5).
 *
 * mu, rho, eta: per-node maps (N each). fs: 3N (component-major) or NULL.
 * g: envelope table g(t_n), n < n_g (0 beyond). v0: 3N initial velocity or NULL;
 * the start is u^0 = 0, u^{-1} = -dt v0 (m applied), i.e. udot^0 = v0.
 * sensors: 3*ns node indices (i, j, k). traces: [n_steps][ns][3], entry n holds
 * u^{n+1} at each sensor. u_out / uprev_out (3N each, nullable) receive
 * u^{n_steps} and u^{n_steps-1}. u_in / uprev_in (3N each, nullable) override
 * the start state (u^0, u^{-1}) for restart tests. divform != 0 replaces
 * (mu/rho) L u and (eta/rho) L udot by (1/rho) K_mu u and (1/rho) K_eta udot.
 */
/* Divergence-form operator (variant of Sec. 3.1 for heterogeneous media):
 * (K_kappa q)_i = sum over the six faces of kappa_f (q_nb - q_i) / dx^2 with the
 * face coefficient kappa_f = (kappa_i + kappa_nb) / 2; interior nodes only. */
static void div_form(int nx, int ny, int nz, double dx, const double *kap, const double *q, double *out)
{
    const double inv = 1.0 / (dx * dx);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(i, j, k);
                if (!is_interior(i, j, k, nx, ny, nz)) {
                    out[c] = 0.0;
                    continue;
                }
                const size_t nb[6] = {IDX(i - 1, j, k), IDX(i + 1, j, k), IDX(i, j - 1, k),
                                      IDX(i, j + 1, k), IDX(i, j, k - 1), IDX(i, j, k + 1)};
                double s = 0.0;
                for (int f = 0; f < 6; ++f) s += 0.5 * (kap[c] + kap[nb[f]]) * (q[nb[f]] - q[c]);
                out[c] = s * inv;
            }
}

int or_run(int nx, int ny, int nz, double dx, double dt, const double *mu, const double *rho,
           const double *eta, const double *fs, const double *g, int n_g, const double *v0,
           const double *u_in, const double *uprev_in, int n_steps, const int *sensors, int ns,
           double *traces, double *u_out, double *uprev_out, int divform)
{
    size_t N = (size_t)nx * ny * nz;
    double *um = (double *)calloc(3 * N, sizeof(double)); /* u^{n-1} */
    double *u0 = (double *)calloc(3 * N, sizeof(double)); /* u^n     */
    double *up = (double *)calloc(3 * N, sizeof(double)); /* u^{n+1} */
    double *w = (double *)calloc(3 * N, sizeof(double));  /* udot^n  */
    double *lu = (double *)calloc(N, sizeof(double));
    double *lw = (double *)calloc(N, sizeof(double));
    if (!um || !u0 || !up || !w || !lu || !lw) {
        free(um); free(u0); free(up); free(w); free(lu); free(lw);
        return -1;
    }
    if (u_in) memcpy(u0, u_in, 3 * N * sizeof(double));
    if (uprev_in) memcpy(um, uprev_in, 3 * N * sizeof(double));
    if (v0 && !uprev_in)
        #pragma omp parallel for schedule(static)
        for (size_t c = 0; c < 3 * N; ++c) um[c] = u0[c] - dt * v0[c];
    for (int c = 0; c < 3; ++c) {
        apply_mask(nx, ny, nz, u0 + c * N);
        apply_mask(nx, ny, nz, um + c * N);
    }

    for (int n = 0; n < n_steps; ++n) {
        const double gn = (g && n < n_g) ? g[n] : 0.0;
        #pragma omp parallel for schedule(static)
        for (size_t c = 0; c < 3 * N; ++c) w[c] = (u0[c] - um[c]) / dt;
        for (int comp = 0; comp < 3; ++comp) {
            const double *uc = u0 + comp * N;
            const double *ucm = um + comp * N;
            double *ucp = up + comp * N;
            if (divform) {  /* lu = K_mu u, lw = K_eta udot (coefficients inside) */
                div_form(nx, ny, nz, dx, mu, uc, lu);
                div_form(nx, ny, nz, dx, eta, w + comp * N, lw);
            } else {
                or_laplacian(nx, ny, nz, dx, uc, lu);
                or_laplacian(nx, ny, nz, dx, w + comp * N, lw);
            }
#pragma omp parallel for schedule(static)
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        size_t c = IDX(i, j, k);
                        if (!is_interior(i, j, k, nx, ny, nz)) {
                            ucp[c] = 0.0;
                            continue;
                        }
                        double a = divform ? (lu[c] + lw[c]) / rho[c]
                                           : (mu[c] / rho[c]) * lu[c] + (eta[c] / rho[c]) * lw[c];
                        if (fs) a += (gn / rho[c]) * fs[comp * N + c];
                        ucp[c] = 2.0 * uc[c] - ucm[c] + dt * dt * a;
                    }
        }
        if (traces)
            for (int s = 0; s < ns; ++s) {
                size_t c = IDX(sensors[3 * s], sensors[3 * s + 1], sensors[3 * s + 2]);
                for (int comp = 0; comp < 3; ++comp)
                    traces[((size_t)n * ns + s) * 3 + comp] = up[comp * N + c];
            }
        double *t = um;
        um = u0;
        u0 = up;
        up = t;
    }
    if (u_out) memcpy(u_out, u0, 3 * N * sizeof(double));
    if (uprev_out) memcpy(uprev_out, um, 3 * N * sizeof(double));
    free(um); free(u0); free(up); free(w); free(lu); free(lw);
    return 0;
}

/*
 * 1D restriction of the same recurrence (Sec. 4.3 harmonic benchmark): a chain
 * of n nodes, u_0^n = amp r(t_n) sin(omega t_n) driven (Dirichlet), u_{n-1} = 0,
 * r(t) = (1 - cos(pi t / t_ramp)) / 2 for t < t_ramp, else 1 (t_ramp <= 0: r = 1),
 *   u_i^{n+1} = 2u_i^n - u_i^{n-1}
 *             + dt^2 [ (mu/rho) D2 u^n + (eta/rho) D2 (u^n - u^{n-1})/dt ]_i.
 * Records u at the sensor nodes for every step: rec[step][s] holds u^{step+1}.
 */
int or_kv1d_run(int n, double dx, double dt, double mu, double rho, double eta, double omega,
                double amp, double t_ramp, int n_steps, const int *sensors, int ns, double *rec)
{
    double *um = (double *)calloc(n, sizeof(double));
    double *u0 = (double *)calloc(n, sizeof(double));
    double *up = (double *)calloc(n, sizeof(double));
    if (!um || !u0 || !up) {
        free(um); free(u0); free(up);
        return -1;
    }
    const double inv = 1.0 / (dx * dx);
    for (int s = 0; s < n_steps; ++s) {
        for (int i = 1; i < n - 1; ++i) {
            double lu = (u0[i + 1] - 2.0 * u0[i] + u0[i - 1]) * inv;
            double wp = (u0[i + 1] - um[i + 1]) / dt;
            double wc = (u0[i] - um[i]) / dt;
            double wm = (u0[i - 1] - um[i - 1]) / dt;
            double lw = (wp - 2.0 * wc + wm) * inv;
            double a = (mu / rho) * lu + (eta / rho) * lw;
            up[i] = 2.0 * u0[i] - um[i] + dt * dt * a;
        }
        const double tn = (double)(s + 1) * dt;
        const double ramp = (t_ramp > 0.0 && tn < t_ramp) ? 0.5 * (1.0 - cos(M_PI * tn / t_ramp)) : 1.0;
        up[0] = amp * ramp * sin(omega * tn);
        up[n - 1] = 0.0;
        for (int q = 0; q < ns; ++q) rec[(size_t)s * ns + q] = up[sensors[q]];
        double *t = um;
        um = u0;
        u0 = up;
        up = t;
    }
    free(um); free(u0); free(up);
    return 0;
}

/*
 * Direct-loop 3D convolution (test infrastructure for the learned warm start;
 * no counterpart in the paper's method). Channel-last tensors [z][y][x][C],
 * 3x3x3 taps t = (dz+1)*9 + (dy+1)*3 + (dx+1), zero padding of one voxel,
 * weights W[t][ci][co]:
 *   out[v][co] = bias[co] + sum_{t, ci} in[v + d(t)][ci] W[t][ci][co]
 * and the two gradients of a scalar loss with upstream gradient g = dL/dout:
 *   gin[v][ci]  = sum_{t, co} g[v - d(t)][co] W[t][ci][co]
 *   gW[t][ci][co] = sum_v in[v + d(t)][ci] g[v][co],   gb[co] = sum_v g[v][co]
 */
void or_conv3d_fwd(int nx, int ny, int nz, int cin, int cout, const double *in, const double *W,
                   const double *bias, double *out)
{
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int co = 0; co < cout; ++co) {
                    double s = bias ? bias[co] : 0.0;
                    for (int t = 0; t < 27; ++t) {
                        const int xx = x + t % 3 - 1, yy = y + (t / 3) % 3 - 1, zz = z + t / 9 - 1;
                        if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
                        const double *a = in + (((size_t)zz * ny + yy) * nx + xx) * cin;
                        for (int ci = 0; ci < cin; ++ci) s += a[ci] * W[((size_t)t * cin + ci) * cout + co];
                    }
                    out[(((size_t)z * ny + y) * nx + x) * cout + co] = s;
                }
}

void or_conv3d_bwd(int nx, int ny, int nz, int cin, int cout, const double *in, const double *W,
                   const double *g, double *gin, double *gW, double *gb)
{
    const size_t V = (size_t)nx * ny * nz;
    if (gin) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x)
                    for (int ci = 0; ci < cin; ++ci) {
                        double s = 0.0;
                        for (int t = 0; t < 27; ++t) {
                            const int xx = x - (t % 3 - 1), yy = y - ((t / 3) % 3 - 1), zz = z - (t / 9 - 1);
                            if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
                            const double *gg = g + (((size_t)zz * ny + yy) * nx + xx) * cout;
                            for (int co = 0; co < cout; ++co) s += gg[co] * W[((size_t)t * cin + ci) * cout + co];
                        }
                        gin[(((size_t)z * ny + y) * nx + x) * cin + ci] = s;
                    }
    }
    if (gW) {
#pragma omp parallel for schedule(static)
        for (int t = 0; t < 27; ++t)
            for (int ci = 0; ci < cin; ++ci)
                for (int co = 0; co < cout; ++co) {
                    double s = 0.0;
                    for (int z = 0; z < nz; ++z)
                        for (int y = 0; y < ny; ++y)
                            for (int x = 0; x < nx; ++x) {
                                const int xx = x + t % 3 - 1, yy = y + (t / 3) % 3 - 1, zz = z + t / 9 - 1;
                                if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
                                s += in[(((size_t)zz * ny + yy) * nx + xx) * cin + ci] *
                                     g[(((size_t)z * ny + y) * nx + x) * cout + co];
                            }
                    gW[((size_t)t * cin + ci) * cout + co] = s;
                }
    }
    if (gb)
        for (int co = 0; co < cout; ++co) {
            double s = 0.0;
            for (size_t v = 0; v < V; ++v) s += g[v * cout + co];
            gb[co] = s;
        }
}
