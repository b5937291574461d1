/*
 * fdoracle.c -- plain, slow, FP64 CPU oracle for the explicit
 * finite-difference wave solvers of Louboutin et al., "Performance
 * prediction of finite-difference solvers for different computer
 * architectures" (arXiv 1608.03984).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it. The GPU library shares no
 * code, header, table or constant with this file; it derives its own
 * weights and coefficients.
 *
 * Conventions (all arrays are dense, x fastest):
 *   computational grid nx*ny*nz (physical grid plus nb sponge points on
 *   every face), index (k*ny + j)*nx + i, i along x, j along y, k along z
 *   (depth). Points outside the grid read as 0 (zero Dirichlet ghosts) or,
 *   when `periodic` is set (closed-form tests only), wrap around.
 *   Physical coordinate of computational index i is (i - nb)*h metres.
 *
 * Every function cites the passage of the paper it restates. Readings of
 * passages the paper leaves open are marked READING.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "fdoracle.h"

#define MAXR 16

typedef struct {
    int nx, ny, nz, r, periodic;
    double h;
    double w2[MAXR + 1]; /* second-derivative weights at offsets 0..r */
    double c1[MAXR + 1]; /* first-derivative weights at offsets 0..r (c1[0]=0) */
} grid_t;

/* ------------------------------------------------------------------------- */
/* Finite-difference weights                                                 */
/* ------------------------------------------------------------------------- */

/*
 * Weights of the derivatives 0..mmax at point z from values at the nodes
 * x[0..n], by Fornberg's recursion (B. Fornberg, "Generation of finite
 * difference formulas on arbitrarily spaced grids", Math. Comp. 51, 1988).
 * out[(node)*(mmax+1) + m] is the weight of node `node` in the m-th
 * derivative. The paper's "1D symmetric stencil of size k" (Section
 * "Stencil operators") is this formula on the k = 2r+1 nodes -r..r.
 */
int or_fornberg(int n, const double *x, double z, int mmax, double *out)
{
    if (n < 0 || mmax < 0 || !x || !out) return -1;
    const int M = mmax + 1;
    memset(out, 0, sizeof(double) * (size_t)(n + 1) * (size_t)M);
    double prod_prev = 1.0;
    double dz_prev = x[0] - z;
    out[0] = 1.0;
    for (int i = 1; i <= n; ++i) {
        const int mtop = i < mmax ? i : mmax;
        double prod = 1.0;
        const double dz_last = dz_prev;
        dz_prev = x[i] - z;
        for (int j = 0; j < i; ++j) {
            const double dx = x[i] - x[j];
            prod *= dx;
            if (j == i - 1) {
                /* the new node i, built from node i-1's previous weights */
                for (int m = mtop; m >= 1; --m)
                    out[i * M + m] = prod_prev *
                        (m * out[(i - 1) * M + m - 1] - dz_last * out[(i - 1) * M + m]) / prod;
                out[i * M + 0] = -prod_prev * dz_last * out[(i - 1) * M + 0] / prod;
            }
            /* update of the older node j */
            for (int m = mtop; m >= 1; --m)
                out[j * M + m] = (dz_prev * out[j * M + m] - m * out[j * M + m - 1]) / dx;
            out[j * M + 0] = dz_prev * out[j * M + 0] / dx;
        }
        prod_prev = prod;
    }
    return 0;
}

/*
 * Central weights of the first and second derivative of space order
 * `order` = 2r on the 2r+1 nodes -r..r (Section "Stencil operators":
 * fixed support of size k = order+1 for every derivative).
 * w2[m], c1[m] are the weights at offset +m, m = 0..r (the weight at -m is
 * w2[m], resp. -c1[m]). Unit grid spacing.
 */
int or_fd_weights(int order, double *w2, double *c1)
{
    if (order < 2 || order > 2 * MAXR || (order & 1)) return -1;
    const int r = order / 2, n = 2 * r;
    double x[2 * MAXR + 1];
    double W[(2 * MAXR + 1) * 3];
    for (int m = -r; m <= r; ++m) x[m + r] = (double)m;
    if (or_fornberg(n, x, 0.0, 2, W)) return -1;
    for (int m = 0; m <= r; ++m) {
        if (w2) w2[m] = W[(m + r) * 3 + 2];
        if (c1) c1[m] = W[(m + r) * 3 + 1];
    }
    if (c1) c1[0] = 0.0;
    return 0;
}

static int grid_init(grid_t *g, int nx, int ny, int nz, int order, double h, int periodic)
{
    if (nx < 1 || ny < 1 || nz < 1 || h <= 0.0) return -1;
    g->nx = nx; g->ny = ny; g->nz = nz; g->h = h; g->periodic = periodic;
    g->r = order / 2;
    return or_fd_weights(order, g->w2, g->c1);
}

static inline long gidx(const grid_t *g, long i, long j, long k)
{
    return (k * g->ny + j) * (long)g->nx + i;
}

/* value at (i,j,k); zero outside the grid unless periodic */
static inline double val(const grid_t *g, const double *u, long i, long j, long k)
{
    if (g->periodic) {
        i = ((i % g->nx) + g->nx) % g->nx;
        j = ((j % g->ny) + g->ny) % g->ny;
        k = ((k % g->nz) + g->nz) % g->nz;
    } else if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz) {
        return 0.0;
    }
    return u[gidx(g, i, j, k)];
}

/* unit step along axis a (0=x, 1=y, 2=z) */
static inline void axis_step(int a, long s, long *di, long *dj, long *dk)
{
    *di = a == 0 ? s : 0;
    *dj = a == 1 ? s : 0;
    *dk = a == 2 ? s : 0;
}

/* d^2u/dx_a^2 at (i,j,k): the k-point second-derivative stencil / h^2 */
static double d2(const grid_t *g, const double *u, long i, long j, long k, int a)
{
    double s = g->w2[0] * val(g, u, i, j, k);
    for (int m = 1; m <= g->r; ++m) {
        long di, dj, dk;
        axis_step(a, m, &di, &dj, &dk);
        s += g->w2[m] * (val(g, u, i + di, j + dj, k + dk) + val(g, u, i - di, j - dj, k - dk));
    }
    return s / (g->h * g->h);
}

/*
 * d^2u/dx_a dx_b (a != b) at (i,j,k): tensor product of the k-point
 * first-derivative stencils along a and b, / h^2.
 * READING: the paper fixes the support ("fixed support for all
 * derivatives", Section "Stencil operators") and the count of
 * multiplications (k^2-2k) but not the taps; the tensor product of the
 * central first-derivative stencils is the stencil with that support.
 */
static double dab(const grid_t *g, const double *u, long i, long j, long k, int a, int b)
{
    double s = 0.0;
    for (int m = 1; m <= g->r; ++m) {
        for (int n = 1; n <= g->r; ++n) {
            long ai, aj, ak, bi, bj, bk;
            axis_step(a, m, &ai, &aj, &ak);
            axis_step(b, n, &bi, &bj, &bk);
            const double q =
                  val(g, u, i + ai + bi, j + aj + bj, k + ak + bk)
                - val(g, u, i + ai - bi, j + aj - bj, k + ak - bk)
                - val(g, u, i - ai + bi, j - aj + bj, k - ak + bk)
                + val(g, u, i - ai - bi, j - aj - bj, k - ak - bk);
            s += g->c1[m] * g->c1[n] * q;
        }
    }
    return s / (g->h * g->h);
}

/* du/dx_a at (i,j,k): central first-derivative stencil / h */
static double d1(const grid_t *g, const double *u, long i, long j, long k, int a)
{
    double s = 0.0;
    for (int m = 1; m <= g->r; ++m) {
        long di, dj, dk;
        axis_step(a, m, &di, &dj, &dk);
        s += g->c1[m] * (val(g, u, i + di, j + dj, k + dk) - val(g, u, i - di, j - dj, k - dk));
    }
    return s / g->h;
}

/* ------------------------------------------------------------------------- */
/* Single operators (exported for the closed-form tests)                     */
/* ------------------------------------------------------------------------- */

/* out = Laplacian of u, sum of the three second-derivative stencils
 * (Eq. Acou, the operator of the acoustic stencil) */
int or_laplacian(int nx, int ny, int nz, int order, double h, int periodic,
                 const double *u, double *out)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz, order, h, periodic)) return -1;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i)
                out[gidx(&g, i, j, k)] = d2(&g, u, i, j, k, 0) + d2(&g, u, i, j, k, 1) + d2(&g, u, i, j, k, 2);
    return 0;
}

/* out = derivative of u: which = 0,1,2 -> d/dx,d/dy,d/dz; 3,4,5 -> d2/dx2,
 * d2/dy2, d2/dz2; 6,7,8 -> d2/dxdy, d2/dxdz, d2/dydz (Section "Stencil
 * operators", the three derivative types of Table 1) */
int or_derivative(int nx, int ny, int nz, int order, double h, int periodic, int which,
                  const double *u, double *out)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz, order, h, periodic)) return -1;
    if (which < 0 || which > 8) return -1;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                double v;
                switch (which) {
                case 0: case 1: case 2: v = d1(&g, u, i, j, k, which); break;
                case 3: case 4: case 5: v = d2(&g, u, i, j, k, which - 3); break;
                case 6: v = dab(&g, u, i, j, k, 0, 1); break;
                case 7: v = dab(&g, u, i, j, k, 0, 2); break;
                default: v = dab(&g, u, i, j, k, 1, 2); break;
                }
                out[gidx(&g, i, j, k)] = v;
            }
    return 0;
}

/*
 * The three rotated operators of Eq. DiffOp applied to u at every point,
 * with the trigonometric factors of the local tilt theta and azimuth phi
 * written exactly as in Eq. DiffOp.
 * READING: the printed G_yy carries "sin(2 phi)^2 d2/dxdy"; with the
 * rotated axis ybar = (-sin phi, cos phi, 0) the coefficient is
 * -sin(2 phi) (unsquared), which is what makes Gxx+Gyy+Gzz the Laplacian.
 */
static void rotated_ops(const grid_t *g, const double *u, long i, long j, long k,
                        double th, double ph, double *Gxx, double *Gyy, double *Gzz)
{
    const double dxx = d2(g, u, i, j, k, 0), dyy = d2(g, u, i, j, k, 1), dzz = d2(g, u, i, j, k, 2);
    const double dxy = dab(g, u, i, j, k, 0, 1), dxz = dab(g, u, i, j, k, 0, 2), dyz = dab(g, u, i, j, k, 1, 2);
    const double ct = cos(th), st = sin(th), cp = cos(ph), sp = sin(ph);
    const double s2t = sin(2.0 * th), s2p = sin(2.0 * ph);
    if (Gxx)
        *Gxx = cp * cp * ct * ct * dxx + sp * sp * ct * ct * dyy + st * st * dzz
             + s2p * ct * ct * dxy - sp * s2t * dyz - cp * s2t * dxz;
    if (Gyy)
        *Gyy = sp * sp * dxx + cp * cp * dyy - s2p * dxy;
    if (Gzz)
        *Gzz = cp * cp * st * st * dxx + sp * sp * st * st * dyy + ct * ct * dzz
             + s2p * st * st * dxy + sp * s2t * dyz + cp * s2t * dxz;
}

/* out_x/out_y/out_z = G_xbarxbar u, G_ybarybar u, G_zbarzbar u (Eq. DiffOp);
 * theta/phi per point in radians. Any output may be NULL. */
int or_rotated(int nx, int ny, int nz, int order, double h, int periodic,
               const double *theta, const double *phi, const double *u,
               double *out_x, double *out_y, double *out_z)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz, order, h, periodic)) return -1;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                const long p = gidx(&g, i, j, k);
                double a, b, c;
                rotated_ops(&g, u, i, j, k, theta[p], phi[p], &a, &b, &c);
                if (out_x) out_x[p] = a;
                if (out_y) out_y[p] = b;
                if (out_z) out_z[p] = c;
            }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Sponge                                                                    */
/* ------------------------------------------------------------------------- */

/*
 * READING (the paper leaves absorbing boundaries out of its model, Section
 * "Introduction to stencil computation"): damped wave equation
 * m u_tt + m gamma u_t - lap u = q with gamma = g(i) + g(j) + g(k), each a
 * linear ramp over the nb sponge points of its axis, from 0 at the first
 * sponge point's inner neighbour to gamma_max at the outermost point.
 * gamma_max = 3 vmax ln(1/R) / (2 nb h).
 */
double or_sponge_gamma_max(double vmax, int nb, double h, double R)
{
    if (nb <= 0) return 0.0;
    return 3.0 * vmax * log(1.0 / R) / (2.0 * nb * h);
}

int or_sponge_profile(int n_comp, int nb, double gamma_max, double *out)
{
    if (n_comp < 1 || nb < 0 || 2 * nb > n_comp) return -1;
    const int n_phys = n_comp - 2 * nb;
    for (int i = 0; i < n_comp; ++i) {
        int d = 0;
        if (i < nb) d = nb - i;
        else if (i > nb + n_phys - 1) d = i - (nb + n_phys - 1);
        out[i] = nb > 0 ? gamma_max * (double)d / (double)nb : 0.0;
    }
    return 0;
}

/* P = 1 + gamma dt/2 and Q = 1 - gamma dt/2 at point (i,j,k) */
static inline void damping(const double *gx, const double *gy, const double *gz, double dt,
                           long i, long j, long k, double *P, double *Q)
{
    const double gh = (gx ? gx[i] : 0.0) + (gy ? gy[j] : 0.0) + (gz ? gz[k] : 0.0);
    *P = 1.0 + 0.5 * dt * gh;
    *Q = 1.0 - 0.5 * dt * gh;
}

/* ------------------------------------------------------------------------- */
/* Sparse points: trilinear injection and interpolation                      */
/* ------------------------------------------------------------------------- */

/*
 * The 8 trilinear corners and weights of a point at physical position
 * (x,y,z) metres. Returns the number of corners inside the grid (corners
 * outside are dropped). READING: the paper only says the source is added
 * after the stencil (Algorithm 1); off-grid points are spread trilinearly.
 */
static int corners(const grid_t *g, int nb, const double *xyz, long *idx, double *w)
{
    const double f[3] = { xyz[0] / g->h + nb, xyz[1] / g->h + nb, xyz[2] / g->h + nb };
    long b[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        b[a] = (long)floor(f[a]);
        t[a] = f[a] - (double)b[a];
    }
    int n = 0;
    for (int c = 0; c < 8; ++c) {
        const long i = b[0] + (c & 1), j = b[1] + ((c >> 1) & 1), k = b[2] + ((c >> 2) & 1);
        const double wt = ((c & 1) ? t[0] : 1.0 - t[0]) * (((c >> 1) & 1) ? t[1] : 1.0 - t[1])
                        * (((c >> 2) & 1) ? t[2] : 1.0 - t[2]);
        if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz) continue;
        idx[n] = gidx(g, i, j, k);
        w[n] = wt;
        ++n;
    }
    return n;
}

/* traces[rec] = trilinear interpolation of u at each receiver */
int or_interpolate(int nx, int ny, int nz, double h, int nb, const double *u,
                   int nrec, const double *rec_xyz, double *traces)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz, 2, h, 0)) return -1;
    for (int r = 0; r < nrec; ++r) {
        long idx[8];
        double w[8];
        const int n = corners(&g, nb, rec_xyz + 3 * r, idx, w);
        double s = 0.0;
        for (int c = 0; c < n; ++c) s += w[c] * u[idx[c]];
        traces[r] = s;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Acoustic time step (Algorithm 1 with Eq. Acou)                            */
/* ------------------------------------------------------------------------- */

/*
 * One step of Algorithm 1 for Eq. Acou with the sponge READING:
 *   P u+ = 2u - Q u- + c (lap u + q),   c = dt^2 v^2 = dt^2/m,
 * i.e. the central second difference of u_tt plus a central first
 * difference for the damping term. The source term q_n (Algorithm 1 "Add
 * Source", after the stencil) is the discrete delta of each source,
 * trilinear weight / h^3, times its amplitude amp[s] at this step.
 * up may not alias u; it may alias um.
 */
static void acoustic_update(const grid_t *g, const double *u, const double *um, const double *c,
                            const double *gx, const double *gy, const double *gz, double dt,
                            double *up)
{
#pragma omp parallel for schedule(static)
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                const long p = gidx(g, i, j, k);
                const double lap = d2(g, u, i, j, k, 0) + d2(g, u, i, j, k, 1) + d2(g, u, i, j, k, 2);
                double P, Q;
                damping(gx, gy, gz, dt, i, j, k, &P, &Q);
                up[p] = (2.0 * u[p] - Q * um[p] + c[p] * lap) / P;
            }
}

/* "Add Source": u+ += c q / P at the corners of every source */
static void add_source(const grid_t *g, int nb, const double *c, const double *gx,
                       const double *gy, const double *gz, double dt,
                       int nsrc, const double *src_xyz, const double *amp, double scale,
                       double *up)
{
    for (int s = 0; s < nsrc; ++s) {
        long idx[8];
        double w[8];
        const int n = corners(g, nb, src_xyz + 3 * s, idx, w);
        for (int q = 0; q < n; ++q) {
            const long p = idx[q];
            const long i = p % g->nx, j = (p / g->nx) % g->ny, k = p / ((long)g->nx * g->ny);
            double P, Q;
            damping(gx, gy, gz, dt, i, j, k, &P, &Q);
            up[p] += c[p] * w[q] * amp[s] * scale / P;
        }
    }
}

int or_acoustic_step(int nx, int ny, int nz, int order, double h, int periodic, int nb,
                     double dt, const double *c, const double *gx, const double *gy,
                     const double *gz, const double *u, const double *um,
                     int nsrc, const double *src_xyz, const double *amp, double *up)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz, order, h, periodic)) return -1;
    if (up == u) return -1;
    acoustic_update(&g, u, um, c, gx, gy, gz, dt, up);
    if (nsrc > 0) add_source(&g, nb, c, gx, gy, gz, dt, nsrc, src_xyz, amp, 1.0 / (h * h * h), up);
    return 0;
}

/*
 * nt steps of Algorithm 1 from u_0 = u_-1 = 0 (Eq. Acou initial state).
 * Step n uses the wavelet row n (wavelet[n*nsrc + s], the amplitude at
 * t_n = n dt) and produces u_{n+1}; traces[(n+1)*nrec + r] records
 * u_{n+1} at receiver r, traces[r] = 0 (READING: nt+1 samples, d[0] = u_0).
 * u_out/um_out (may be NULL) receive u_nt and u_{nt-1}. When `history`
 * is non-NULL it receives u_0..u_nt ((nt+1) fields).
 */
int or_acoustic_forward(int nx, int ny, int nz, int order, double h, int nb, double dt,
                        const double *c, const double *gx, const double *gy, const double *gz,
                        int nsrc, const double *src_xyz, const double *wavelet, int nt,
                        int nrec, const double *rec_xyz, double *traces,
                        double *u_out, double *um_out, double *history)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz, order, h, 0) || nt < 0) return -1;
    const long N = (long)nx * ny * nz;
    double *a = calloc((size_t)N, sizeof(double));  /* u_{n-1} */
    double *b = calloc((size_t)N, sizeof(double));  /* u_n     */
    double *amp = malloc(sizeof(double) * (size_t)(nsrc > 0 ? nsrc : 1));
    if (!a || !b || !amp) { free(a); free(b); free(amp); return -2; }
    if (traces && nrec > 0) memset(traces, 0, sizeof(double) * (size_t)nrec);
    if (history) memset(history, 0, sizeof(double) * (size_t)N);
    for (int n = 0; n < nt; ++n) {
        for (int s = 0; s < nsrc; ++s) amp[s] = wavelet[(long)n * nsrc + s];
        /* u_{n+1} overwrites u_{n-1} */
        acoustic_update(&g, b, a, c, gx, gy, gz, dt, a);
        if (nsrc > 0) add_source(&g, nb, c, gx, gy, gz, dt, nsrc, src_xyz, amp, 1.0 / (h * h * h), a);
        double *t = a; a = b; b = t;   /* b = u_{n+1}, a = u_n */
        if (traces && nrec > 0) or_interpolate(nx, ny, nz, h, nb, b, nrec, rec_xyz, traces + (long)(n + 1) * nrec);
        if (history) memcpy(history + (long)(n + 1) * N, b, sizeof(double) * (size_t)N);
    }
    if (u_out) memcpy(u_out, b, sizeof(double) * (size_t)N);
    if (um_out) memcpy(um_out, a, sizeof(double) * (size_t)N);
    free(a); free(b); free(amp);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* TTI time step (Eq. TTI with Eq. DiffOp)                                   */
/* ------------------------------------------------------------------------- */

/*
 * One step of Eq. TTI:
 *   P p+ = 2p - Q p- + c [ (1+2 eps)(Gxx+Gyy) p + sqrt(1+2 delta) Gzz r + q ]
 *   P r+ = 2r - Q r- + c [ sqrt(1+2 delta)(Gxx+Gyy) p + Gzz r + q ]
 * with the same damping READING as the acoustic step. READING: the same
 * source q enters both equations, as printed. eps, delta, theta, phi are
 * per point (angles in radians). pp/rp may alias pm/rm.
 */
static void tti_update(const grid_t *g, const double *p, const double *pm, const double *r,
                       const double *rm, const double *c, const double *eps, const double *delta,
                       const double *theta, const double *phi, const double *gx, const double *gy,
                       const double *gz, double dt, double *pp, double *rp)
{
#pragma omp parallel for schedule(static)
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                const long q = gidx(g, i, j, k);
                double Gxx_p, Gyy_p, Gzz_r;
                rotated_ops(g, p, i, j, k, theta[q], phi[q], &Gxx_p, &Gyy_p, NULL);
                rotated_ops(g, r, i, j, k, theta[q], phi[q], NULL, NULL, &Gzz_r);
                const double e = 1.0 + 2.0 * eps[q];
                const double d = sqrt(1.0 + 2.0 * delta[q]);
                double P, Q;
                damping(gx, gy, gz, dt, i, j, k, &P, &Q);
                const double hp = Gxx_p + Gyy_p;
                const double np_ = (2.0 * p[q] - Q * pm[q] + c[q] * (e * hp + d * Gzz_r)) / P;
                const double nr_ = (2.0 * r[q] - Q * rm[q] + c[q] * (d * hp + Gzz_r)) / P;
                pp[q] = np_;
                rp[q] = nr_;
            }
}

int or_tti_step(int nx, int ny, int nz, int order, double h, int periodic, int nb, double dt,
                const double *c, const double *eps, const double *delta, const double *theta,
                const double *phi, const double *gx, const double *gy, const double *gz,
                const double *p, const double *pm, const double *r, const double *rm,
                int nsrc, const double *src_xyz, const double *amp, double *pp, double *rp)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz, order, h, periodic)) return -1;
    if (pp == p || rp == r || pp == r || rp == p) return -1;
    tti_update(&g, p, pm, r, rm, c, eps, delta, theta, phi, gx, gy, gz, dt, pp, rp);
    if (nsrc > 0) {
        add_source(&g, nb, c, gx, gy, gz, dt, nsrc, src_xyz, amp, 1.0 / (h * h * h), pp);
        add_source(&g, nb, c, gx, gy, gz, dt, nsrc, src_xyz, amp, 1.0 / (h * h * h), rp);
    }
    return 0;
}

/*
 * nt TTI steps from zero state; receivers record p (READING: the paper
 * does not say which field is recorded). Outputs as or_acoustic_forward;
 * fields_out (may be NULL) receives p_nt, p_{nt-1}, r_nt, r_{nt-1}.
 */
int or_tti_forward(int nx, int ny, int nz, int order, double h, int nb, double dt,
                   const double *c, const double *eps, const double *delta, const double *theta,
                   const double *phi, const double *gx, const double *gy, const double *gz,
                   int nsrc, const double *src_xyz, const double *wavelet, int nt,
                   int nrec, const double *rec_xyz, double *traces, double *fields_out)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz, order, h, 0) || nt < 0) return -1;
    const long N = (long)nx * ny * nz;
    double *pa = calloc((size_t)N, sizeof(double)), *pb = calloc((size_t)N, sizeof(double));
    double *ra = calloc((size_t)N, sizeof(double)), *rb = calloc((size_t)N, sizeof(double));
    double *amp = malloc(sizeof(double) * (size_t)(nsrc > 0 ? nsrc : 1));
    if (!pa || !pb || !ra || !rb || !amp) {
        free(pa); free(pb); free(ra); free(rb); free(amp);
        return -2;
    }
    if (traces && nrec > 0) memset(traces, 0, sizeof(double) * (size_t)nrec);
    for (int n = 0; n < nt; ++n) {
        for (int s = 0; s < nsrc; ++s) amp[s] = wavelet[(long)n * nsrc + s];
        tti_update(&g, pb, pa, rb, ra, c, eps, delta, theta, phi, gx, gy, gz, dt, pa, ra);
        if (nsrc > 0) {
            add_source(&g, nb, c, gx, gy, gz, dt, nsrc, src_xyz, amp, 1.0 / (h * h * h), pa);
            add_source(&g, nb, c, gx, gy, gz, dt, nsrc, src_xyz, amp, 1.0 / (h * h * h), ra);
        }
        double *t = pa; pa = pb; pb = t;
        t = ra; ra = rb; rb = t;
        if (traces && nrec > 0) or_interpolate(nx, ny, nz, h, nb, pb, nrec, rec_xyz, traces + (long)(n + 1) * nrec);
    }
    if (fields_out) {
        memcpy(fields_out, pb, sizeof(double) * (size_t)N);
        memcpy(fields_out + N, pa, sizeof(double) * (size_t)N);
        memcpy(fields_out + 2 * N, rb, sizeof(double) * (size_t)N);
        memcpy(fields_out + 3 * N, ra, sizeof(double) * (size_t)N);
    }
    free(pa); free(pb); free(ra); free(rb); free(amp);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint and FWI gradient of the acoustic recurrence                       */
/* ------------------------------------------------------------------------- */

/*
 * The paper motivates the solvers by FWI/RTM (Introduction) but gives no
 * adjoint; this is the exact transpose of the discrete recurrence above.
 *
 * Forward (n = 0..nt-1):  P u_{n+1} = (2 + C L) u_n - Q u_{n-1} + C q_n,
 *                         d_n = R u_n (n = 0..nt),
 * with C = diag(c), L the symmetric Laplacian matrix, R trilinear
 * interpolation. For J = sum_n <res_n, d_n> (res given), the multipliers
 * mu_k = C lambda_k satisfy, for k = nt..1 with mu_{nt+1} = mu_{nt+2} = 0,
 *     P mu_k = (2 + C L) mu_{k+1} - Q mu_{k+2} + C R^T res_k,
 * i.e. the forward step run backwards, the residual spread with the
 * trilinear weights (no 1/h^3) onto the level being produced. Then
 *     dJ/dwavelet[n][s] = sum_corners w/h^3 mu_{n+1}     (source side)
 *     dJ/dc  = sum_{n=0}^{nt-1} mu_{n+1} (P u_{n+1} - 2 u_n + Q u_{n-1}) / c^2
 *     dJ/dm  = -(1/dt^2) sum_{n} mu_{n+1} (P u_{n+1} - 2 u_n + Q u_{n-1})
 * (c = dt^2/m). `history` holds u_0..u_nt from or_acoustic_forward.
 * Outputs (any may be NULL): wavelet_adj [nt][nsrc], grad_m [N].
 */
int or_acoustic_adjoint(int nx, int ny, int nz, int order, double h, int nb, double dt,
                        const double *c, const double *gx, const double *gy, const double *gz,
                        int nrec, const double *rec_xyz, const double *res, int nt,
                        int nsrc, const double *src_xyz, double *wavelet_adj,
                        const double *history, double *grad_m)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz, order, h, 0) || nt < 0) return -1;
    if (grad_m && !history) return -1;
    const long N = (long)nx * ny * nz;
    double *m2 = calloc((size_t)N, sizeof(double));  /* mu_{k+2} */
    double *m1 = calloc((size_t)N, sizeof(double));  /* mu_{k+1} */
    if (!m2 || !m1) { free(m2); free(m1); return -2; }
    if (grad_m) memset(grad_m, 0, sizeof(double) * (size_t)N);
    if (wavelet_adj && nsrc > 0) memset(wavelet_adj, 0, sizeof(double) * (size_t)nt * nsrc);
    for (int k = nt; k >= 1; --k) {
        /* mu_k overwrites mu_{k+2} */
        acoustic_update(&g, m1, m2, c, gx, gy, gz, dt, m2);
        if (nrec > 0) add_source(&g, nb, c, gx, gy, gz, dt, nrec, rec_xyz, res + (long)k * nrec, 1.0, m2);
        double *t = m2; m2 = m1; m1 = t;   /* m1 = mu_k, m2 = mu_{k+1} */
        const int n = k - 1;               /* mu_k = mu_{n+1} */
        if (wavelet_adj && nsrc > 0) {
            for (int s = 0; s < nsrc; ++s) {
                long idx[8];
                double w[8];
                const int nc = corners(&g, nb, src_xyz + 3 * s, idx, w);
                double acc = 0.0;
                for (int q = 0; q < nc; ++q) acc += w[q] * m1[idx[q]];
                wavelet_adj[(long)n * nsrc + s] = acc / (h * h * h);
            }
        }
        if (grad_m) {
            const double *un1 = history + (long)(n + 1) * N;
            const double *un = history + (long)n * N;
            const double *unm = n >= 1 ? history + (long)(n - 1) * N : NULL;
#pragma omp parallel for schedule(static)
            for (long kk = 0; kk < nz; ++kk)
                for (long j = 0; j < ny; ++j)
                    for (long i = 0; i < nx; ++i) {
                        const long p = gidx(&g, i, j, kk);
                        double P, Q;
                        damping(gx, gy, gz, dt, i, j, kk, &P, &Q);
                        const double sec = P * un1[p] - 2.0 * un[p] + Q * (unm ? unm[p] : 0.0);
                        grad_m[p] -= m1[p] * sec / (dt * dt);
                    }
        }
    }
    free(m2); free(m1);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Learned closure: a small 3x3x3 convolutional network                      */
/* ------------------------------------------------------------------------- */

/*
 * The paper has no learned component (its cost-benefit section trades grid
 * spacing against stencil order); the closure corrects a coarse low-order
 * step toward the fine high-order one. Network: conv 3 -> H, ReLU,
 * conv H -> H, ReLU, conv H -> 1, all 3x3x3 "valid" convolutions (each
 * shrinks the box by one point per face):
 *   out[co][z][y][x] = b[co] + sum_ci sum_{a,b,c in 0..2}
 *                      W[co][ci][(a*3+b)*3+c] in[ci][z+a][y+b][x+c].
 * Parameters, concatenated: W1[H][3][27], b1[H], W2[H][H][27], b2[H],
 * W3[1][H][27], b3[1].
 */
static void conv_valid(int ci, int co, int nz, int ny, int nx, const double *in, const double *w,
                       const double *b, int relu, double *out)
{
    const int oz = nz - 2, oy = ny - 2, ox = nx - 2;
    for (int o = 0; o < co; ++o)
        for (int z = 0; z < oz; ++z)
            for (int y = 0; y < oy; ++y)
                for (int x = 0; x < ox; ++x) {
                    double s = b[o];
                    for (int i = 0; i < ci; ++i)
                        for (int a = 0; a < 3; ++a)
                            for (int bb = 0; bb < 3; ++bb)
                                for (int c = 0; c < 3; ++c)
                                    s += w[((long)o * ci + i) * 27 + (a * 3 + bb) * 3 + c] *
                                         in[(((long)i * nz + z + a) * ny + y + bb) * nx + x + c];
                    out[(((long)o * oz + z) * oy + y) * ox + x] = (relu && s < 0.0) ? 0.0 : s;
                }
}

/* d(loss)/d(in) and d(loss)/d(w, b) of conv_valid, given g = d(loss)/d(out)
 * (after the ReLU mask of the layer's own output has been applied). */
static void conv_valid_backward(int ci, int co, int nz, int ny, int nx, const double *in,
                                const double *w, const double *g, double *gin, double *gw,
                                double *gb)
{
    const int oz = nz - 2, oy = ny - 2, ox = nx - 2;
    if (gin) memset(gin, 0, sizeof(double) * (size_t)ci * nz * ny * nx);
    for (int o = 0; o < co; ++o)
        for (int z = 0; z < oz; ++z)
            for (int y = 0; y < oy; ++y)
                for (int x = 0; x < ox; ++x) {
                    const double gv = g[(((long)o * oz + z) * oy + y) * ox + x];
                    gb[o] += gv;
                    for (int i = 0; i < ci; ++i)
                        for (int a = 0; a < 3; ++a)
                            for (int bb = 0; bb < 3; ++bb)
                                for (int c = 0; c < 3; ++c) {
                                    const long t = ((long)o * ci + i) * 27 + (a * 3 + bb) * 3 + c;
                                    const long p = (((long)i * nz + z + a) * ny + y + bb) * nx + x + c;
                                    gw[t] += gv * in[p];
                                    if (gin) gin[p] += gv * w[t];
                                }
                }
}

long or_closure_num_params(int H)
{
    return (long)H * 3 * 27 + H + (long)H * H * 27 + H + (long)H * 27 + 1;
}

/*
 * Forward pass of one sample: in [3][nz][ny][nx] -> out [nz-6][ny-6][nx-6].
 * a1 [H][nz-2]..., a2 [H][nz-4]... receive the (post-ReLU) activations
 * when non-NULL.
 */
int or_closure_forward(int H, int nz, int ny, int nx, const double *params, const double *in,
                       double *a1, double *a2, double *out)
{
    if (H < 1 || nz < 7 || ny < 7 || nx < 7) return -1;
    const double *W1 = params, *b1 = W1 + (long)H * 3 * 27, *W2 = b1 + H, *b2 = W2 + (long)H * H * 27,
                 *W3 = b2 + H, *b3 = W3 + (long)H * 27;
    const long n1 = (long)H * (nz - 2) * (ny - 2) * (nx - 2), n2 = (long)H * (nz - 4) * (ny - 4) * (nx - 4);
    double *t1 = a1 ? a1 : malloc(sizeof(double) * n1);
    double *t2 = a2 ? a2 : malloc(sizeof(double) * n2);
    if (!t1 || !t2) return -2;
    conv_valid(3, H, nz, ny, nx, in, W1, b1, 1, t1);
    conv_valid(H, H, nz - 2, ny - 2, nx - 2, t1, W2, b2, 1, t2);
    conv_valid(H, 1, nz - 4, ny - 4, nx - 4, t2, W3, b3, 0, out);
    if (!a1) free(t1);
    if (!a2) free(t2);
    return 0;
}

/*
 * Mean-squared error of a batch and its gradient w.r.t. the parameters:
 * loss = (1/M) sum over samples and output points of (out - target)^2,
 * M = batch * (nz-6)(ny-6)(nx-6). in [batch][3][nz][ny][nx], target
 * [batch][nz-6][ny-6][nx-6]; grad (may be NULL) receives d loss / d params.
 */
int or_closure_loss_grad(int H, int batch, int nz, int ny, int nx, const double *params,
                         const double *in, const double *target, double *loss, double *grad)
{
    if (batch < 1) return -1;
    const long np_ = or_closure_num_params(H);
    const double *W2 = params + (long)H * 3 * 27 + H, *W3 = W2 + (long)H * H * 27 + H;
    double *gW1 = grad, *gb1 = grad ? gW1 + (long)H * 3 * 27 : NULL, *gW2 = grad ? gb1 + H : NULL,
           *gb2 = grad ? gW2 + (long)H * H * 27 : NULL, *gW3 = grad ? gb2 + H : NULL,
           *gb3 = grad ? gW3 + (long)H * 27 : NULL;
    if (grad) memset(grad, 0, sizeof(double) * np_);
    const long s0 = (long)nz * ny * nx, s1 = (long)(nz - 2) * (ny - 2) * (nx - 2),
               s2 = (long)(nz - 4) * (ny - 4) * (nx - 4), s3 = (long)(nz - 6) * (ny - 6) * (nx - 6);
    double *a1 = malloc(sizeof(double) * H * s1), *a2 = malloc(sizeof(double) * H * s2);
    double *out = malloc(sizeof(double) * s3), *g3 = malloc(sizeof(double) * s3);
    double *g2 = malloc(sizeof(double) * H * s2), *g1 = malloc(sizeof(double) * H * s1);
    if (!a1 || !a2 || !out || !g3 || !g2 || !g1) return -2;
    const double M = (double)batch * s3;
    double L = 0.0;
    for (int b = 0; b < batch; ++b) {
        or_closure_forward(H, nz, ny, nx, params, in + b * 3 * s0, a1, a2, out);
        for (long p = 0; p < s3; ++p) {
            const double r = out[p] - target[b * s3 + p];
            L += r * r / M;
            g3[p] = 2.0 * r / M;
        }
        if (!grad) continue;
        conv_valid_backward(H, 1, nz - 4, ny - 4, nx - 4, a2, W3, g3, g2, gW3, gb3);
        for (long p = 0; p < H * s2; ++p)
            if (a2[p] <= 0.0) g2[p] = 0.0;  /* ReLU of layer 2 */
        conv_valid_backward(H, H, nz - 2, ny - 2, nx - 2, a1, W2, g2, g1, gW2, gb2);
        for (long p = 0; p < H * s1; ++p)
            if (a1[p] <= 0.0) g1[p] = 0.0;  /* ReLU of layer 1 */
        conv_valid_backward(3, H, nz, ny, nx, in + b * 3 * s0, params, g1, NULL, gW1, gb1);
    }
    if (loss) *loss = L;
    free(a1); free(a2); free(out); free(g3); free(g2); free(g1);
    return 0;
}
