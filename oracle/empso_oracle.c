/*
 * FP64 CPU oracle for the EMPSO fitness-evaluation path (arXiv 1905.12795).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with
 * the CUDA library: every formula here is restated from the paper (or from the
 * textbook it relies on) in the plainest form, with no blocking, fusion or
 * reordering beyond what the definition states.
 *
 * Build: gcc -O2 -ffp-contract=off -std=c11 -fPIC -shared -pthread.  FMA
 * contraction is off so that the same operation sequence gives the same bits
 * on x86-64 and aarch64 hosts.
 *
 * Contents (paper sections in brackets):
 *   - centred 2nd-derivative coefficients, orders 2/4/8   ["Testing approach":
 *     2nd order in time, 8th order in space]
 *   - Ricker wavelet                                       ["Testing approach"]
 *   - time axis from the CFL limit, damping-layer profile ["Algorithm overview",
 *     JSON nbpml; the damping law itself is a reading, the paper is silent]
 *   - natural cubic spline / bilinear two-grid interpolation ["Testing approach",
 *     two-grid strategy]
 *   - one explicit time step, one shot gather, the L2 misfit ["Testing approach"]
 *   - Philox4x32-10 counter RNG, Box-Muller normal with project-written log/cos
 *   - PSO Eq. 1-3 with velocity clamp (JSON lambda), box constraint, gbest
 *     topology and elitist mutation (EMPSO figure)          ["Theory"]
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Finite-difference coefficients                                            */
/* ------------------------------------------------------------------------ */

/* Central second-derivative weights c_0..c_R of accuracy order 2R (Fornberg
 * 1988 tables): f''(x) ~ (1/h^2) [c_0 f(x) + sum_m c_m (f(x+mh) + f(x-mh))].
 * The paper's modelling uses order 8 in space and its local FWI order 16
 * ("Testing approach"); orders 2 and 4 are kept for the smaller workloads.
 * Returns R, or -1 for an unsupported order. */
int eo_fd_coeffs(int order, double *c)
{
    if (order == 2) {
        c[0] = -2.0; c[1] = 1.0;
        return 1;
    }
    if (order == 4) {
        c[0] = -5.0 / 2.0; c[1] = 4.0 / 3.0; c[2] = -1.0 / 12.0;
        return 2;
    }
    if (order == 8) {
        c[0] = -205.0 / 72.0; c[1] = 8.0 / 5.0; c[2] = -1.0 / 5.0;
        c[3] = 8.0 / 315.0; c[4] = -1.0 / 560.0;
        return 4;
    }
    if (order == 16) {   /* the local FWI's spatial order ("Testing approach") */
        c[0] = -1077749.0 / 352800.0; c[1] = 16.0 / 9.0; c[2] = -14.0 / 45.0;
        c[3] = 112.0 / 1485.0; c[4] = -7.0 / 396.0; c[5] = 112.0 / 32175.0;
        c[6] = -2.0 / 3861.0; c[7] = 16.0 / 315315.0; c[8] = -1.0 / 411840.0;
        return 8;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Source wavelet and time axis                                              */
/* ------------------------------------------------------------------------ */

/* Ricker wavelet of peak frequency f0, delayed by 1/f0 ("Testing approach":
 * Ricker source; the JSON example's f0 key).  r(t) = (1 - 2 pi^2 f0^2 tau^2)
 * exp(-pi^2 f0^2 tau^2), tau = t - 1/f0. */
double eo_ricker(double f0, double t)
{
    double tau = t - 1.0 / f0;
    double a = M_PI * M_PI * f0 * f0 * tau * tau;
    return (1.0 - 2.0 * a) * exp(-a);
}

/* Time axis: dt_max = 2 / (vmax sqrt(rho (1/hx^2 + 1/hz^2))) with
 * rho = |c_0 + 2 sum_m (-1)^m c_m| (the largest eigenvalue of the 1-D
 * stencil, reached by the checkerboard mode).  nt = ceil(T / (cfl dt_max)) + 1
 * and dt = T / (nt - 1), so that T is an exact multiple of dt.  Returns nt. */
int eo_time_axis(int order, double hx, double hz, double vmax, double T,
                 double cfl, double *dt_out)
{
    double c[9];
    int R = eo_fd_coeffs(order, c);
    if (R < 0) return -1;
    double rho = c[0];
    for (int m = 1; m <= R; ++m) rho += 2.0 * ((m % 2) ? -c[m] : c[m]);
    rho = fabs(rho);
    double dtmax = 2.0 / (vmax * sqrt(rho * (1.0 / (hx * hx) + 1.0 / (hz * hz))));
    int nt = (int)ceil(T / (cfl * dtmax)) + 1;
    *dt_out = T / (double)(nt - 1);
    return nt;
}

/* Damping coefficient eta along one axis of a padded line of n + 2 pad nodes
 * (JSON nbpml = pad).  eta(d) = eta_max (d / L)^2 with d the distance in metres
 * from the inner edge of the layer, L = pad h and
 * eta_max = 3 vmax ln(1/R) / (2 L), R = 1e-3 (Collino & Tsogka 2001). */
void eo_damping_profile(int n, int pad, double h, double vmax, double *eta)
{
    int N = n + 2 * pad;
    double L = pad * h;
    for (int I = 0; I < N; ++I) {
        double d = 0.0;
        if (I < pad) d = (double)(pad - I) * h;
        else if (I > pad + n - 1) d = (double)(I - (pad + n - 1)) * h;
        eta[I] = 0.0;
        if (pad > 0 && d > 0.0) {
            double etamax = 3.0 * vmax * log(1.0 / 1e-3) / (2.0 * L);
            eta[I] = etamax * (d / L) * (d / L);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Spatial operator and one time step                                        */
/* ------------------------------------------------------------------------ */

/* 2-D Laplacian of order `order` on an NZ x NX grid stored row-major
 * (x fastest), with u = 0 outside the grid. */
void eo_laplacian(const double *u, int NX, int NZ, double hx, double hz,
                  int order, double *out)
{
    double c[9];
    int R = eo_fd_coeffs(order, c);
    for (int J = 0; J < NZ; ++J) {
        for (int I = 0; I < NX; ++I) {
            double sx = c[0] * u[(size_t)J * NX + I];
            double sz = c[0] * u[(size_t)J * NX + I];
            for (int m = 1; m <= R; ++m) {
                double l = (I - m >= 0) ? u[(size_t)J * NX + (I - m)] : 0.0;
                double r = (I + m < NX) ? u[(size_t)J * NX + (I + m)] : 0.0;
                double t = (J - m >= 0) ? u[(size_t)(J - m) * NX + I] : 0.0;
                double b = (J + m < NZ) ? u[(size_t)(J + m) * NX + I] : 0.0;
                sx += c[m] * (l + r);
                sz += c[m] * (t + b);
            }
            out[(size_t)J * NX + I] = sx / (hx * hx) + sz / (hz * hz);
        }
    }
}

/* One step of the damped, constant-density acoustic equation
 *   u_tt + eta u_t = v^2 (lap u + s)
 * centred in time (2nd order): with a = v^2 dt^2,
 *   u1 = [2 u0 - (1 - eta dt/2) um + a (lap u0 + s)] / (1 + eta dt/2).
 * eta = etax[I] + etaz[J].  `s` may be NULL (no source).  `work` holds NX*NZ
 * doubles. */
void eo_step(const double *um, const double *u0, double *u1, const double *vel,
             const double *etax, const double *etaz, const double *s,
             int NX, int NZ, double hx, double hz, int order, double dt,
             double *work)
{
    eo_laplacian(u0, NX, NZ, hx, hz, order, work);
    for (int J = 0; J < NZ; ++J) {
        for (int I = 0; I < NX; ++I) {
            size_t k = (size_t)J * NX + I;
            double a = vel[k] * vel[k] * dt * dt;
            double eta = etax[I] + etaz[J];
            double src = s ? s[k] : 0.0;
            double num = 2.0 * u0[k] - (1.0 - eta * dt / 2.0) * um[k] + a * (work[k] + src);
            u1[k] = num / (1.0 + eta * dt / 2.0);
        }
    }
}

/* Bilinear weights of a point (x, z) in metres on the padded grid, whose node
 * (I, J) sits at ((I - pad) hx, (J - pad) hz).  Fills the four corner indices
 * and weights.  The lower corner is kept at most at NX-2 / NZ-2 so that all
 * four corners are inside the grid. */
static void bilinear_corners(double x, double z, int pad, double hx, double hz,
                             int NX, int NZ, int *I0, int *J0, double w[4])
{
    double fx = x / hx + pad, fz = z / hz + pad;
    int i0 = (int)floor(fx), j0 = (int)floor(fz);
    if (i0 > NX - 2) i0 = NX - 2;
    if (j0 > NZ - 2) j0 = NZ - 2;
    if (i0 < 0) i0 = 0;
    if (j0 < 0) j0 = 0;
    double ax = fx - i0, az = fz - j0;
    w[0] = (1.0 - ax) * (1.0 - az); /* (i0,   j0)   */
    w[1] = ax * (1.0 - az);         /* (i0+1, j0)   */
    w[2] = (1.0 - ax) * az;         /* (i0,   j0+1) */
    w[3] = ax * az;                 /* (i0+1, j0+1) */
    *I0 = i0;
    *J0 = j0;
}

/* Grid description shared by the shot routines. */
typedef struct {
    int nx, nz, pad, order;
    double hx, hz, dt, f0, vmax_damp;
    int nt;
} eo_grid;

/* One shot gather ("Testing approach": FD modelling of each shot, L2 misfit).
 *
 * vel: physical velocity model [nz][nx] (m/s), edge-extended here into the
 * damping pad.  Source at (sx, sz) injected bilinearly as a point density
 * r(t_n) b / (hx hz) into step n; receiver r records the bilinear sample of
 * u^{n+1} after step n, so trace sample n is the field at t_{n+1}.
 * u^{-1} = u^0 = 0.  Writes traces [nt][nrec] if `traces` is non-NULL and
 * returns phi = 1/2 sum_n sum_r (d - dobs)^2 if `dobs` is non-NULL (else 0). */
double eo_shot(const eo_grid *g, const double *vel, double sx, double sz,
               const double *rec_xz, int nrec, const double *dobs,
               double *traces)
{
    int NX = g->nx + 2 * g->pad, NZ = g->nz + 2 * g->pad;
    size_t N = (size_t)NX * NZ;
    double *vp = malloc(N * sizeof(double));
    double *um = calloc(N, sizeof(double));
    double *u0 = calloc(N, sizeof(double));
    double *u1 = calloc(N, sizeof(double));
    double *s = calloc(N, sizeof(double));
    double *work = malloc(N * sizeof(double));
    double *etax = malloc(NX * sizeof(double));
    double *etaz = malloc(NZ * sizeof(double));
    eo_damping_profile(g->nx, g->pad, g->hx, g->vmax_damp, etax);
    eo_damping_profile(g->nz, g->pad, g->hz, g->vmax_damp, etaz);
    for (int J = 0; J < NZ; ++J) {
        int j = J - g->pad;
        if (j < 0) j = 0;
        if (j > g->nz - 1) j = g->nz - 1;
        for (int I = 0; I < NX; ++I) {
            int i = I - g->pad;
            if (i < 0) i = 0;
            if (i > g->nx - 1) i = g->nx - 1;
            vp[(size_t)J * NX + I] = vel[(size_t)j * g->nx + i];
        }
    }
    int sI, sJ;
    double sw[4];
    bilinear_corners(sx, sz, g->pad, g->hx, g->hz, NX, NZ, &sI, &sJ, sw);
    int *rI = malloc((nrec > 0 ? nrec : 1) * sizeof(int));
    int *rJ = malloc((nrec > 0 ? nrec : 1) * sizeof(int));
    double *rw = malloc((nrec > 0 ? nrec : 1) * 4 * sizeof(double));
    for (int r = 0; r < nrec; ++r)
        bilinear_corners(rec_xz[2 * r], rec_xz[2 * r + 1], g->pad, g->hx, g->hz,
                         NX, NZ, &rI[r], &rJ[r], &rw[4 * r]);
    double phi = 0.0;
    for (int n = 0; n < g->nt; ++n) {
        double rn = eo_ricker(g->f0, n * g->dt);
        double dens = rn / (g->hx * g->hz);
        s[(size_t)sJ * NX + sI] = dens * sw[0];
        s[(size_t)sJ * NX + sI + 1] = dens * sw[1];
        s[(size_t)(sJ + 1) * NX + sI] = dens * sw[2];
        s[(size_t)(sJ + 1) * NX + sI + 1] = dens * sw[3];
        eo_step(um, u0, u1, vp, etax, etaz, s, NX, NZ, g->hx, g->hz, g->order,
                g->dt, work);
        for (int r = 0; r < nrec; ++r) {
            size_t k = (size_t)rJ[r] * NX + rI[r];
            const double *w = &rw[4 * r];
            double d = w[0] * u1[k] + w[1] * u1[k + 1] + w[2] * u1[k + NX] +
                       w[3] * u1[k + NX + 1];
            if (traces) traces[(size_t)n * nrec + r] = d;
            if (dobs) {
                double e = d - dobs[(size_t)n * nrec + r];
                phi += 0.5 * e * e;
            }
        }
        double *t = um; um = u0; u0 = u1; u1 = t;
    }
    free(vp); free(um); free(u0); free(u1); free(s); free(work);
    free(etax); free(etaz); free(rI); free(rJ); free(rw);
    return phi;
}

/* A batch of (model, shot) instances on one grid, spread over `nthreads`
 * POSIX threads, one instance at a time per thread.  Instance q = m * S + s.
 * Results are written per instance, so thread timing cannot change them. */
typedef struct {
    const eo_grid *g;
    const double *vel;        /* [M][nz][nx] */
    const double *shot_xz;    /* [S][2] */
    const int *rec_begin;     /* [S] */
    const int *rec_count;     /* [S] */
    const double *rec_xz;     /* [*][2] */
    const double *dobs;       /* flat, per shot [nt][nrec_s]; may be NULL */
    const long *dobs_off;     /* [S] offsets into dobs */
    double *traces;           /* flat like dobs but per instance; may be NULL */
    const long *tr_off;       /* [M*S] */
    double *phi;              /* [M*S] */
    int M, S;
    int next;
    pthread_mutex_t lock;
} eo_batch_job;

static void *batch_worker(void *arg)
{
    eo_batch_job *J = (eo_batch_job *)arg;
    size_t cells = (size_t)J->g->nx * J->g->nz;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int q = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (q >= J->M * J->S) break;
        int m = q / J->S, s = q % J->S;
        J->phi[q] = eo_shot(J->g, J->vel + (size_t)m * cells, J->shot_xz[2 * s],
                            J->shot_xz[2 * s + 1], J->rec_xz + 2 * (size_t)J->rec_begin[s],
                            J->rec_count[s], J->dobs ? J->dobs + J->dobs_off[s] : NULL,
                            J->traces ? J->traces + J->tr_off[q] : NULL);
    }
    return NULL;
}

void eo_shot_batch(int nx, int nz, int pad, int order, double hx, double hz,
                   double dt, int nt, double f0, double vmax_damp,
                   const double *vel, int M, const double *shot_xz,
                   const int *rec_begin, const int *rec_count, int S,
                   const double *rec_xz, const double *dobs, const long *dobs_off,
                   double *traces, const long *tr_off, double *phi, int nthreads)
{
    eo_grid g = {nx, nz, pad, order, hx, hz, dt, f0, vmax_damp, nt};
    eo_batch_job J = {&g, vel, shot_xz, rec_begin, rec_count, rec_xz, dobs,
                      dobs_off, traces, tr_off, phi, M, S, 0,
                      PTHREAD_MUTEX_INITIALIZER};
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, batch_worker, &J);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
}

/* ------------------------------------------------------------------------ */
/* Two-grid parameterisation                                                 */
/* ------------------------------------------------------------------------ */

/* Solve the dense n x n system A y = b in place by Gaussian elimination with
 * partial pivoting (A row-major, destroyed; b overwritten by y). */
static void dense_solve(double *A, double *b, int n)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(A[r * n + k]) > fabs(A[p * n + k])) p = r;
        if (p != k) {
            for (int c = 0; c < n; ++c) {
                double t = A[k * n + c]; A[k * n + c] = A[p * n + c]; A[p * n + c] = t;
            }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            double f = A[r * n + k] / A[k * n + k];
            for (int c = k; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
            b[r] -= f * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int c = k + 1; c < n; ++c) s -= A[k * n + c] * b[c];
        b[k] = s / A[k * n + k];
    }
}

/* Interpolation matrix W [n][K] from K control nodes, uniformly spanning grid
 * indices 0..n-1 (node k at xi_k = k (n-1)/(K-1)), to the n grid nodes.
 * mode 0: natural cubic spline (the "bicubic spline" of the tensor product);
 * mode 1: piecewise linear (the paper's bilinear two-grid interpolation,
 * "Testing approach").  Column k is the interpolant of the k-th unit vector.
 * K >= 2. */
void eo_interp_matrix(int K, int n, int mode, double *W)
{
    double H = (double)(n - 1) / (double)(K - 1);
    double *A = malloc(sizeof(double) * K * K);
    double *M = malloc(sizeof(double) * K);
    for (int k = 0; k < K; ++k) {
        /* second derivatives M_j of the natural spline through e_k:
         * M_0 = M_{K-1} = 0 and, for interior j,
         * H/6 M_{j-1} + 2H/3 M_j + H/6 M_{j+1} = (y_{j+1} - 2 y_j + y_{j-1}) / H */
        memset(A, 0, sizeof(double) * K * K);
        for (int j = 0; j < K; ++j) {
            if (j == 0 || j == K - 1 || mode == 1) {
                A[j * K + j] = 1.0;
                M[j] = 0.0;
                continue;
            }
            A[j * K + j - 1] = H / 6.0;
            A[j * K + j] = 2.0 * H / 3.0;
            A[j * K + j + 1] = H / 6.0;
            double yp = (j + 1 == k) ? 1.0 : 0.0;
            double y0 = (j == k) ? 1.0 : 0.0;
            double ym = (j - 1 == k) ? 1.0 : 0.0;
            M[j] = (yp - 2.0 * y0 + ym) / H;
        }
        dense_solve(A, M, K);
        for (int i = 0; i < n; ++i) {
            double xi = (double)i;
            int seg = (int)floor(xi / H);
            if (seg > K - 2) seg = K - 2;
            if (seg < 0) seg = 0;
            double t = (xi - seg * H) / H;
            double y0 = (seg == k) ? 1.0 : 0.0;
            double y1 = (seg + 1 == k) ? 1.0 : 0.0;
            double s = (1.0 - t) * y0 + t * y1 +
                       H * H / 6.0 *
                           (((1.0 - t) * (1.0 - t) * (1.0 - t) - (1.0 - t)) * M[seg] +
                            (t * t * t - t) * M[seg + 1]);
            W[(size_t)i * K + k] = s;
        }
    }
    free(A);
    free(M);
}

/* Velocity model [nz][nx] from the control-node values C [Kz][Kx]
 * (node index k = kz Kx + kx): V = Wz C Wx^T, clipped to [vmin, vmax]. */
void eo_interp_model(const double *C, int Kz, int Kx, int nz, int nx, int mode,
                     double vmin, double vmax, double *V)
{
    double *Wz = malloc(sizeof(double) * nz * Kz);
    double *Wx = malloc(sizeof(double) * nx * Kx);
    eo_interp_matrix(Kz, nz, mode, Wz);
    eo_interp_matrix(Kx, nx, mode, Wx);
    for (int j = 0; j < nz; ++j) {
        for (int i = 0; i < nx; ++i) {
            double v = 0.0;
            for (int kz = 0; kz < Kz; ++kz)
                for (int kx = 0; kx < Kx; ++kx)
                    v += Wz[(size_t)j * Kz + kz] * C[kz * Kx + kx] * Wx[(size_t)i * Kx + kx];
            if (v < vmin) v = vmin;
            if (v > vmax) v = vmax;
            V[(size_t)j * nx + i] = v;
        }
    }
    free(Wz);
    free(Wx);
}

/* Irregular control grid of the paper's "Testing approach" (two-grid
 * strategy with a variable node spacing): L depth levels at z_l (strictly
 * increasing, metres), level l holding n_l nodes at x positions
 * node_x[off_l .. off_l + n_l) (strictly increasing) with values
 * C[off_l ..].  The FD-grid velocity at (x, z) = (i hx, j hz) is the
 * bilinear rule taken level-wise: along each of the two levels bracketing
 * z, linear interpolation in x between that level's neighbouring nodes
 * (the end values held beyond the first/last node), then linear
 * interpolation in z between the two levels (the first/last level held
 * above/below).  Points at depth z <= water_z (when water_z > 0) take the
 * fixed water velocity v_water (the water layer the prior information
 * fixes).  The result is clipped to [vmin, vmax]. */
static double eo_level_profile(const double *xs, const double *cs, int n, double x)
{
    if (n == 1 || x <= xs[0]) return cs[0];
    if (x >= xs[n - 1]) return cs[n - 1];
    int i = 0;
    while (!(x < xs[i + 1])) ++i;
    double a = (x - xs[i]) / (xs[i + 1] - xs[i]);
    return (1.0 - a) * cs[i] + a * cs[i + 1];
}

void eo_interp_levels(int L, const double *level_z, const int *level_n, const double *node_x,
                      const double *C, int nz, int nx, double hx, double hz, double water_z,
                      double v_water, double vmin, double vmax, double *V)
{
    int *off = malloc(sizeof(int) * (L + 1));
    off[0] = 0;
    for (int l = 0; l < L; ++l) off[l + 1] = off[l] + level_n[l];
    for (int j = 0; j < nz; ++j) {
        double z = j * hz;
        int la, lb;
        double b;
        if (z <= level_z[0]) { la = lb = 0; b = 0.0; }
        else if (z >= level_z[L - 1]) { la = lb = L - 1; b = 0.0; }
        else {
            la = 0;
            while (!(z < level_z[la + 1])) ++la;
            lb = la + 1;
            b = (z - level_z[la]) / (level_z[lb] - level_z[la]);
        }
        for (int i = 0; i < nx; ++i) {
            double x = i * hx;
            double va = eo_level_profile(node_x + off[la], C + off[la], level_n[la], x);
            double vb = eo_level_profile(node_x + off[lb], C + off[lb], level_n[lb], x);
            double v = (1.0 - b) * va + b * vb;
            if (water_z > 0.0 && z <= water_z) v = v_water;
            if (v < vmin) v = vmin;
            if (v > vmax) v = vmax;
            V[(size_t)j * nx + i] = v;
        }
    }
    free(off);
}

/* Depth-dependent search ranges ("Testing approach"): the first and last
 * levels get [v (1 - lo), v (1 + hi)] around the prior 1-D velocity v of that
 * level; the limits of every intermediate level lie on the straight lines (in
 * depth) through the first and last levels' minima and maxima.  Every node
 * of a level shares its level's range.  xmin, xmax: [sum n_l]. */
void eo_level_bounds(int L, const double *level_z, const int *level_n, double v_first,
                     double v_last, double lo_first, double hi_first, double lo_last,
                     double hi_last, double *xmin, double *xmax)
{
    double min0 = v_first * (1.0 - lo_first), max0 = v_first * (1.0 + hi_first);
    double min1 = v_last * (1.0 - lo_last), max1 = v_last * (1.0 + hi_last);
    int k = 0;
    for (int l = 0; l < L; ++l) {
        double s = L > 1 ? (level_z[l] - level_z[0]) / (level_z[L - 1] - level_z[0]) : 0.0;
        double lo = min0 + s * (min1 - min0), hi = max0 + s * (max1 - max0);
        for (int i = 0; i < level_n[l]; ++i, ++k) {
            xmin[k] = lo;
            xmax[k] = hi;
        }
    }
}

/* Observed-data preprocessing ("Testing approach": the recorded data are
 * low-pass filtered below the modelling band before the inversion): a
 * band-limited resampling of traces with the Blackman-windowed sinc kernel
 *   h(tau) = 2 fc sinc(2 fc tau) w(tau / W),  sinc(x) = sin(pi x) / (pi x),
 *   w(u) = 0.42 + 0.5 cos(pi u) + 0.08 cos(2 pi u) for |u| < 1, else 0,
 * evaluated at the output times:
 *   out[s][m][r] = dt_in sum_n in[s][n][r] h(m dt_out - n dt_in)
 * (records start at t = 0; samples outside the record count as zero).  With
 * dt_out = dt_in this is a zero-phase low-pass; otherwise it also moves the
 * traces to another time axis. */
static double eo_bsinc(double tau, double fc, double W)
{
    double u = tau / W;
    if (u <= -1.0 || u >= 1.0) return 0.0;
    double w = 0.42 + 0.5 * cos(M_PI * u) + 0.08 * cos(2.0 * M_PI * u);
    double x = 2.0 * fc * tau;
    double sinc = (x == 0.0) ? 1.0 : sin(M_PI * x) / (M_PI * x);
    return 2.0 * fc * sinc * w;
}

void eo_lowpass(const double *in, int S, int nt_in, int nrec, double dt_in, double *out,
                int nt_out, double dt_out, double fc, double W)
{
    for (int s = 0; s < S; ++s)
        for (int m = 0; m < nt_out; ++m)
            for (int r = 0; r < nrec; ++r) {
                double t = m * dt_out, acc = 0.0;
                for (int n = 0; n < nt_in; ++n)
                    acc += in[((size_t)s * nt_in + n) * nrec + r] * eo_bsinc(t - n * dt_in, fc, W);
                out[((size_t)s * nt_out + m) * nrec + r] = dt_in * acc;
            }
}

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers                                              */
/* ------------------------------------------------------------------------ */

/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
 *   (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
 *   c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
 * with the key bumped by the Weyl constants between rounds. */
void eo_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in the open interval (0, 1): w 2^-32 + 2^-33. */
static double u01(uint32_t w) { return (double)w * 0x1p-32 + 0x1p-33; }

/* Natural logarithm written from the series
 *   ln m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), s = (m-1)/(m+1),
 * after the exact split u = m 2^e with m in [sqrt(1/2), sqrt(2)).  Terms up to
 * s^23 (|s| <= 0.1716) leave a truncation error below 1e-18.  Every step is a
 * single IEEE operation in a fixed order. */
double eo_log(double u)
{
    int e;
    double m = frexp(u, &e); /* m in [0.5, 1) */
    if (m < 0.70710678118654752440) {
        m = m * 2.0;
        e = e - 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double s2 = s * s;
    double p = 1.0 / 23.0;
    p = p * s2 + 1.0 / 21.0;
    p = p * s2 + 1.0 / 19.0;
    p = p * s2 + 1.0 / 17.0;
    p = p * s2 + 1.0 / 15.0;
    p = p * s2 + 1.0 / 13.0;
    p = p * s2 + 1.0 / 11.0;
    p = p * s2 + 1.0 / 9.0;
    p = p * s2 + 1.0 / 7.0;
    p = p * s2 + 1.0 / 5.0;
    p = p * s2 + 1.0 / 3.0;
    p = p * s2 + 1.0;
    double lnm = 2.0 * s * p;
    return (double)e * 0.69314718055994530942 + lnm;
}

/* Taylor series of cos and sin on [0, pi/4]: terms to theta^20 / theta^21. */
static double cos_series(double x)
{
    double x2 = x * x;
    double p = 1.0 / 2432902008176640000.0;    /* 1/20! */
    p = -p * x2 + 1.0 / 6402373705728000.0;     /* 1/18! */
    p = -p * x2 + 1.0 / 20922789888000.0;       /* 1/16! */
    p = -p * x2 + 1.0 / 87178291200.0;          /* 1/14! */
    p = -p * x2 + 1.0 / 479001600.0;            /* 1/12! */
    p = -p * x2 + 1.0 / 3628800.0;              /* 1/10! */
    p = -p * x2 + 1.0 / 40320.0;                /* 1/8!  */
    p = -p * x2 + 1.0 / 720.0;                  /* 1/6!  */
    p = -p * x2 + 1.0 / 24.0;                   /* 1/4!  */
    p = -p * x2 + 1.0 / 2.0;                    /* 1/2!  */
    p = -p * x2 + 1.0;
    return p;
}

static double sin_series(double x)
{
    double x2 = x * x;
    double p = 1.0 / 51090942171709440000.0;   /* 1/21! */
    p = -p * x2 + 1.0 / 121645100408832000.0;   /* 1/19! */
    p = -p * x2 + 1.0 / 355687428096000.0;      /* 1/17! */
    p = -p * x2 + 1.0 / 1307674368000.0;        /* 1/15! */
    p = -p * x2 + 1.0 / 6227020800.0;           /* 1/13! */
    p = -p * x2 + 1.0 / 39916800.0;             /* 1/11! */
    p = -p * x2 + 1.0 / 362880.0;               /* 1/9!  */
    p = -p * x2 + 1.0 / 5040.0;                 /* 1/7!  */
    p = -p * x2 + 1.0 / 120.0;                  /* 1/5!  */
    p = -p * x2 + 1.0 / 6.0;                    /* 1/3!  */
    p = -p * x2 + 1.0;
    return x * p;
}

/* cos(2 pi t) for t in (0, 1), by the exact reductions t -> 1 - t (t > 1/2),
 * t -> 1/2 - t with a sign flip (t > 1/4) and cos(2 pi t) = sin(2 pi (1/4 - t))
 * (t > 1/8); each subtraction is exact (Sterbenz). */
double eo_cos2pi(double t)
{
    double sign = 1.0;
    if (t > 0.5) t = 1.0 - t;
    if (t > 0.25) {
        t = 0.5 - t;
        sign = -1.0;
    }
    double r;
    if (t > 0.125) r = sin_series((0.25 - t) * 6.28318530717958647693);
    else r = cos_series(t * 6.28318530717958647693);
    return sign * r;
}

/* Random-number purposes: the fourth Philox counter word. */
enum { EO_INIT_X = 0, EO_INIT_V = 1, EO_U1 = 2, EO_U2 = 3, EO_EM_U = 4, EO_EM_N = 5 };

static void philox_at(uint64_t seed, uint32_t k, uint32_t i, uint32_t d,
                      uint32_t purpose, uint32_t out[4])
{
    uint32_t ctr[4] = {k, i, d, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    eo_philox(ctr, key, out);
}

double eo_uniform(uint64_t seed, uint32_t k, uint32_t i, uint32_t d, uint32_t purpose)
{
    uint32_t w[4];
    philox_at(seed, k, i, d, purpose, w);
    return u01(w[0]);
}

/* Standard normal by Box-Muller from words 0 and 1 of one Philox block. */
double eo_normal(uint64_t seed, uint32_t k, uint32_t i, uint32_t d)
{
    uint32_t w[4];
    philox_at(seed, k, i, d, EO_EM_N, w);
    double u1 = u01(w[0]), u2 = u01(w[1]);
    return sqrt(-2.0 * eo_log(u1)) * eo_cos2pi(u2);
}

/* ------------------------------------------------------------------------ */
/* EMPSO                                                                     */
/* ------------------------------------------------------------------------ */

/* Constriction factor, Eq. 3: chi = 2 / |2 - phi - sqrt(phi^2 - 4 phi)|,
 * phi = c1 + c2 >= 4. */
double eo_chi(double c1, double c2)
{
    double phi = c1 + c2;
    return 2.0 / fabs(2.0 - phi - sqrt(phi * phi - 4.0 * phi));
}

typedef struct {
    int P, D;
    double c1, c2, lambda, p_em, nm_frac;
    int em_start, em_enabled;
    uint64_t seed;
} eo_pso;

static double clip(double x, double lo, double hi)
{
    return x < lo ? lo : (x > hi ? hi : x);
}

/* Swarm initialisation ("Theory": random positions, randomized velocities):
 * x ~ U(xmin, xmax), v ~ U(-vmax, vmax) with vmax = lambda (xmax - xmin)
 * (JSON lambda key).  pbest fitness starts at +inf, generation k at 0. */
void eo_pso_init(const eo_pso *c, const double *xmin, const double *xmax,
                 double *x, double *v, double *p, double *pf, int *g, int *k)
{
    for (int i = 0; i < c->P; ++i) {
        for (int d = 0; d < c->D; ++d) {
            double vr = xmax[d] - xmin[d];
            double vm = c->lambda * vr;
            double ux = eo_uniform(c->seed, 0, i, d, EO_INIT_X);
            double uv = eo_uniform(c->seed, 0, i, d, EO_INIT_V);
            x[(size_t)i * c->D + d] = xmin[d] + ux * vr;
            v[(size_t)i * c->D + d] = vm * (2.0 * uv - 1.0);
            p[(size_t)i * c->D + d] = x[(size_t)i * c->D + d];
        }
        pf[i] = INFINITY;
    }
    *g = 0;
    *k = 0;
}

/* One EMPSO generation after the fitness f of the current positions is
 * known ("Theory", Eq. 1-3 and the EM figure; "Testing approach" for the
 * box constraint):
 *   1. k <- k + 1; non-finite fitness counts as +inf.
 *   2. personal bests: if f_i < pf_i (strict) then pf_i = f_i, p_i = x_i.
 *   3. global best g = argmin pf, ties to the lowest index.
 *   4. if EM is enabled and k >= em_start: ASF = stable ascending sort of f
 *      (or of the rank keys, see below);
 *      its last NM = floor(nm_frac P) entries are the worst particles, whose
 *      positions become x_ld = g_d + 0.1 VR_d randn with probability p_em,
 *      else g_d; their velocities are unchanged.
 *   5. every other particle: Eq. 1 with constriction chi (Eq. 3), velocity
 *      clamped to [-vmax, vmax], Eq. 2, position clamped to [xmin, xmax].
 * `order` receives ASF (P ints) when EM ran, else the identity.
 * `rank_in` (may be NULL) replaces f as the key of the EM sort only: with a
 * surrogate pre-screen, particles that were not modelled carry +inf fitness
 * (no best update) and their predicted misfit as sort key. */
void eo_pso_step(const eo_pso *c, const double *xmin, const double *xmax,
                 const double *f_in, const double *rank_in, double *x, double *v, double *p,
                 double *pf, int *g, int *k, int *order, int *em_ran)
{
    int P = c->P, D = c->D;
    *k = *k + 1;
    double *f = malloc(sizeof(double) * P);
    double *key = malloc(sizeof(double) * P);
    for (int i = 0; i < P; ++i) f[i] = isfinite(f_in[i]) ? f_in[i] : INFINITY;
    for (int i = 0; i < P; ++i) {
        double r = rank_in ? rank_in[i] : f_in[i];
        key[i] = isfinite(r) ? r : INFINITY;
    }
    for (int i = 0; i < P; ++i) {
        if (f[i] < pf[i]) {
            pf[i] = f[i];
            for (int d = 0; d < D; ++d) p[(size_t)i * D + d] = x[(size_t)i * D + d];
        }
    }
    int best = 0;
    for (int i = 1; i < P; ++i)
        if (pf[i] < pf[best]) best = i;
    *g = best;
    const double *gx = p + (size_t)best * D;

    int NM = (int)floor(c->nm_frac * P);
    int em = c->em_enabled && *k >= c->em_start && NM > 0;
    for (int i = 0; i < P; ++i) order[i] = i;
    if (em) {
        /* stable insertion sort by fitness: equal keys keep index order */
        for (int a = 1; a < P; ++a) {
            int cur = order[a];
            int b = a - 1;
            while (b >= 0 && key[order[b]] > key[cur]) {
                order[b + 1] = order[b];
                --b;
            }
            order[b + 1] = cur;
        }
    }
    *em_ran = em;
    char *mut = calloc(P, 1);
    if (em)
        for (int r = P - NM; r < P; ++r) mut[order[r]] = 1;

    double chi = eo_chi(c->c1, c->c2);
    for (int i = 0; i < P; ++i) {
        for (int d = 0; d < D; ++d) {
            size_t id = (size_t)i * D + d;
            double vr = xmax[d] - xmin[d];
            if (mut[i]) {
                double u = eo_uniform(c->seed, *k, i, d, EO_EM_U);
                double xn;
                if (u < c->p_em) xn = gx[d] + 0.1 * vr * eo_normal(c->seed, *k, i, d);
                else xn = gx[d];
                x[id] = clip(xn, xmin[d], xmax[d]);
            } else {
                double vm = c->lambda * vr;
                double u1 = eo_uniform(c->seed, *k, i, d, EO_U1);
                double u2 = eo_uniform(c->seed, *k, i, d, EO_U2);
                double vn = chi * (v[id] + c->c1 * u1 * (p[id] - x[id]) +
                                   c->c2 * u2 * (gx[d] - x[id]));
                vn = clip(vn, -vm, vm);
                v[id] = vn;
                x[id] = clip(x[id] + vn, xmin[d], xmax[d]);
            }
        }
    }
    free(mut);
    free(f);
    free(key);
}
