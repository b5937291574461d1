/*
 * fdoracle.h -- FP64 CPU oracle of the explicit FD wave solvers
 * (arXiv 1608.03984). Test infrastructure only: nothing on the GPU path
 * includes this header. Conventions are stated in fdoracle.c.
 * All functions return 0 on success, negative on bad arguments.
 */
#ifndef FDORACLE_H
#define FDORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

int or_fornberg(int n, const double *x, double z, int mmax, double *out);
int or_fd_weights(int order, double *w2, double *c1);

int or_laplacian(int nx, int ny, int nz, int order, double h, int periodic,
                 const double *u, double *out);
int or_derivative(int nx, int ny, int nz, int order, double h, int periodic, int which,
                  const double *u, double *out);
int or_rotated(int nx, int ny, int nz, int order, double h, int periodic,
               const double *theta, const double *phi, const double *u,
               double *out_x, double *out_y, double *out_z);

double or_sponge_gamma_max(double vmax, int nb, double h, double R);
int or_sponge_profile(int n_comp, int nb, double gamma_max, double *out);

int or_interpolate(int nx, int ny, int nz, double h, int nb, const double *u,
                   int nrec, const double *rec_xyz, double *traces);

int or_acoustic_step(int nx, int ny, int nz, int order, double h, int periodic, int nb,
                     double dt, const double *c, const double *gx, const double *gy,
                     const double *gz, const double *u, const double *um,
                     int nsrc, const double *src_xyz, const double *amp, double *up);
int or_acoustic_forward(int nx, int ny, int nz, int order, double h, int nb, double dt,
                        const double *c, const double *gx, const double *gy, const double *gz,
                        int nsrc, const double *src_xyz, const double *wavelet, int nt,
                        int nrec, const double *rec_xyz, double *traces,
                        double *u_out, double *um_out, double *history);

int or_tti_step(int nx, int ny, int nz, int order, double h, int periodic, int nb, double dt,
                const double *c, const double *eps, const double *delta, const double *theta,
                const double *phi, const double *gx, const double *gy, const double *gz,
                const double *p, const double *pm, const double *r, const double *rm,
                int nsrc, const double *src_xyz, const double *amp, double *pp, double *rp);
int or_tti_forward(int nx, int ny, int nz, int order, double h, int nb, double dt,
                   const double *c, const double *eps, const double *delta, const double *theta,
                   const double *phi, const double *gx, const double *gy, const double *gz,
                   int nsrc, const double *src_xyz, const double *wavelet, int nt,
                   int nrec, const double *rec_xyz, double *traces, double *fields_out);

int or_acoustic_adjoint(int nx, int ny, int nz, int order, double h, int nb, double dt,
                        const double *c, const double *gx, const double *gy, const double *gz,
                        int nrec, const double *rec_xyz, const double *res, int nt,
                        int nsrc, const double *src_xyz, double *wavelet_adj,
                        const double *history, double *grad_m);

long or_closure_num_params(int H);
int or_closure_forward(int H, int nz, int ny, int nx, const double *params, const double *in,
                       double *a1, double *a2, double *out);
int or_closure_loss_grad(int H, int batch, int nz, int ny, int nx, const double *params,
                         const double *in, const double *target, double *loss, double *grad);

#ifdef __cplusplus
}
#endif
#endif
