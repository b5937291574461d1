/*
 * fdwave.h -- C ABI of the GB300 (sm_103a) explicit finite-difference wave
 * solver: the time-stepping hot path analysed in Louboutin et al.,
 * "Performance prediction of finite-difference solvers for different
 * computer architectures" (arXiv 1608.03984).
 *
 * What one step computes (Algorithm 1 "Time-stepping", Eq. Acou / Eq. TTI):
 *   acoustic:  P u+ = 2u - Q u- + c (lap u + q)
 *   TTI:       P p+ = 2p - Q p- + c [(1+2e)(Gxx+Gyy) p + sqrt(1+2d) Gzz r + q]
 *              P r+ = 2r - Q r- + c [sqrt(1+2d)(Gxx+Gyy) p + Gzz r + q]
 * with c = dt^2 v^2, the rotated operators of Eq. DiffOp, space order 2..16
 * star stencils (Section "Stencil operators"), P, Q = 1 +- gamma dt/2 the
 * linear sponge (the paper leaves boundaries out; this is the library's
 * choice, fused in the update), q the trilinear point sources divided by
 * h^3 ("Add Source" of Algorithm 1), followed by trilinear receiver
 * interpolation of the new level into FP64 traces.
 *
 * Grids. The caller gives the PHYSICAL grid nx*ny*nz (x fastest, z depth)
 * and spacing h in metres; the library adds nb sponge points on every face
 * (computational grid (nx+2nb)*(ny+2nb)*(nz+2nb)). Outside the
 * computational grid the wavefield is zero. Positions are (x, y, z) metres
 * with the first physical point at the origin; they may lie anywhere in the
 * computational grid, sponge included (else FDW_ERR_OUT_OF_DOMAIN).
 *
 * Memory and streams. Every call is ordered on the CUDA stream given at
 * creation (NULL = the legacy default stream). The library owns its device
 * buffers (allocated with cudaMalloc in fdw_create / fdw_set_* and freed in
 * fdw_destroy). Pointer arguments are caller-owned and only read or written
 * during the call; `ptr_is_device` says whether they are device pointers
 * (copied stream-ordered) or host pointers (the call synchronises the
 * stream before it returns). Calls on one solver are not thread-safe.
 *
 * Errors. Every int-returning call returns FDW_OK (0) or a negative
 * FDW_ERR_* code and leaves a message for fdw_last_error() (thread-local).
 * Device-side failures (a bounded wait in a kernel that gave up, a
 * non-finite wavefield found by fdw_check) are reported by the next
 * synchronising call. No C++ exception crosses this interface.
 */
#ifndef FDWAVE_H
#define FDWAVE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDW_OK 0
#define FDW_ERR_INVALID_ARG (-1)
#define FDW_ERR_UNSTABLE_DT (-2)
#define FDW_ERR_OOM (-3)
#define FDW_ERR_CUDA (-4)
#define FDW_ERR_STATE (-5)         /* call out of order (e.g. step before set_dt) */
#define FDW_ERR_DIVERGED (-6)      /* non-finite wavefield */
#define FDW_ERR_OUT_OF_DOMAIN (-7) /* source/receiver outside the grid */
#define FDW_ERR_DEVICE_TIMEOUT (-8) /* a kernel's bounded wait gave up */

typedef struct fdw_solver fdw_solver;

/* equation */
#define FDW_ACOUSTIC 0 /* Eq. Acou */
#define FDW_TTI 1      /* Eq. TTI with Eq. DiffOp (VTI is theta = phi = 0) */

/* storage type of wavefields and medium parameters; arithmetic is FP32 */
#define FDW_F32 0
#define FDW_BF16 1
#define FDW_F16 2

/* Thread-local message of the last failing call ("" if none). */
const char *fdw_last_error(void);

/* Library version string. */
const char *fdw_version(void);

/*
 * Create a solver. space_order: even, 2..16 (stencil width k = order+1,
 * Section "Stencil operators"). nb >= 0 sponge points per face. stream: a
 * cudaStream_t or NULL. Allocates the wavefield and medium buffers on the
 * current CUDA device. *out receives the handle.
 * Errors: INVALID_ARG (sizes, order, equation, storage), OOM, CUDA.
 */
int fdw_create(fdw_solver **out, int nx, int ny, int nz, double h, int nb, int equation,
               int space_order, int storage, void *stream);

/* Free every buffer of the solver (synchronises its stream). NULL is a no-op. */
int fdw_destroy(fdw_solver *s);

/*
 * Set the medium from PHYSICAL-grid arrays [nz][ny][nx] float32: vp in m/s
 * (> 0); for TTI also eps, delta (Thomsen parameters, eps >= delta >= 0
 * recommended for stability), theta (tilt) and phi (azimuth) in radians;
 * pass NULL for those with the acoustic equation. The sponge points take
 * the value of the nearest physical point. Invalidates dt (call
 * fdw_set_dt again). With BF16/FP16 storage the TTI axis is stored as two
 * components (nx, ny) and nz rebuilt, whose rounding error grows as the
 * axis tips over: tilts beyond 75 degrees are rejected for 16-bit storage
 * (FP32 storage takes any tilt). Errors: INVALID_ARG (NULL vp, vp <= 0 or
 * non-finite, a tilt beyond 75 degrees with 16-bit TTI storage), CUDA.
 */
int fdw_set_model(fdw_solver *s, const float *vp, const float *eps, const float *delta,
                  const float *theta, const float *phi, int ptr_is_device);

/*
 * Largest stable time step of Eq. stability (CFL): vmax dt / h <= sqrt(4/a2),
 * a2 the sum of |weights| of the 3D Laplacian stencil; for TTI vmax is the
 * largest vp sqrt(1+2 eps). Returns a negative value before fdw_set_model.
 */
double fdw_max_stable_dt(const fdw_solver *s);

/*
 * Sponge strength: gamma_max = 3 vref ln(1/R) / (2 nb h) (linear ramp over
 * the nb points of each face). vref <= 0 (the default) uses the model's
 * largest velocity; a fixed vref keeps the damping independent of the model
 * (for gradients w.r.t. the model). Default R = 1e-3. Takes effect at the
 * next fdw_set_dt (dt is marked unset). Errors: INVALID_ARG.
 */
int fdw_set_sponge(fdw_solver *s, double vref, double R);

/*
 * Storage scale S: the buffers hold S times the physical wavefield (the
 * equations are linear, so this only moves the values within the storage
 * type's range). Sources are injected times S; traces, fdw_get_wavefield,
 * fdw_set_wavefield, the adjoint and the gradient undo it, so every value
 * a caller sees is physical. scale = 0 (default) chooses at fdw_set_dt:
 * for FP16 storage the power of two that makes the stored increment of a
 * unit source about 256 (the far field then stays in FP16's normal range),
 * otherwise 1. Set it before stepping (stored levels are not rescaled);
 * dt is marked unset. fdw_get_field_scale returns the scale in use.
 * Errors: INVALID_ARG (scale < 0 or non-finite).
 */
int fdw_set_field_scale(fdw_solver *s, double scale);
double fdw_get_field_scale(const fdw_solver *s);

/*
 * Set dt (seconds): computes c = dt^2 v^2 and the sponge damping.
 * Errors: UNSTABLE_DT if dt > fdw_max_stable_dt, STATE before set_model.
 */
int fdw_set_dt(fdw_solver *s, double dt);

/*
 * Point sources: xyz [nsrc][3] metres (host), wavelet [nt][nsrc] float32
 * (amplitude at t_n = n dt; step n injects row n, steps n >= nt inject
 * nothing). nsrc = 0 clears the sources. Errors: INVALID_ARG, OUT_OF_DOMAIN.
 */
int fdw_set_sources(fdw_solver *s, int nsrc, const double *xyz, const float *wavelet, int nt,
                    int ptr_is_device);

/*
 * Receivers: xyz [nrec][3] metres (host); traces of nt+1 rows are kept on
 * the device in FP64, row n = interpolation of level n (row 0 of a fresh
 * run is 0). For TTI the receivers record p. Clears the traces.
 */
int fdw_set_receivers(fdw_solver *s, int nrec, const double *xyz, int nt);

/* Zero the wavefields, the traces and the step counter (fresh run). */
int fdw_reset(fdw_solver *s);

/* Current step index n (the state holds levels n and n-1). */
int fdw_current_step(const fdw_solver *s);

/*
 * Advance nsteps steps (asynchronous on the stream): stencil update with
 * fused sponge, source injection, receiver interpolation, per step.
 * Errors: STATE (no dt), INVALID_ARG (nsteps < 0), CUDA.
 */
int fdw_step(fdw_solver *s, int nsteps);

/*
 * Copy the traces [(nt+1)][nrec] FP64 into out (host or device).
 * Synchronises when out is a host pointer; reports device timeouts.
 */
int fdw_gather_receivers(fdw_solver *s, double *out, int ptr_is_device);

/*
 * Copy one wavefield level of the computational grid, as float32
 * [(nz+2nb)][(ny+2nb)][(nx+2nb)], into out (host or device).
 * field: 0 = u (acoustic) / p (TTI), 1 = r (TTI); level: 0 = n, 1 = n-1.
 */
int fdw_get_wavefield(const fdw_solver *s, int field, int level, float *out, int ptr_is_device);

/*
 * Overwrite one wavefield level (same layout as fdw_get_wavefield); values
 * are rounded to the storage type. Used for checkpoints and one-step checks.
 */
int fdw_set_wavefield(fdw_solver *s, int field, int level, const float *in, int ptr_is_device);

/* Set the step counter n (after restoring wavefields with fdw_set_wavefield). */
int fdw_set_current_step(fdw_solver *s, int n);

/*
 * Synchronise the stream, report a device timeout flag, and when
 * check_finite is non-zero scan the current levels for NaN/Inf
 * (FDW_ERR_DIVERGED).
 */
int fdw_check(fdw_solver *s, int check_finite);

/*
 * Kernel variant of the stencil update: 0 = the 2.5D z-marching TMA
 * kernel (default), 1 = a one-thread-per-point kernel computing the same
 * step from plain global loads (an independent GPU formulation kept for
 * cross-checks). Errors: INVALID_ARG.
 */
int fdw_set_kernel_variant(fdw_solver *s, int variant);

/*
 * Number of CTAs along z of the 2.5D kernel (each marches nz_comp/zchunks
 * planes); 0 restores the default chosen from the grid size. fdw_get_zchunks
 * returns the value in use (-1 for NULL).
 */
int fdw_set_zchunks(fdw_solver *s, int zchunks);

/*
 * Tile configuration of the 2.5D kernel: acoustic (points per thread in x/y,
 * warps per CTA, z unrolling, planes per CTA barrier; acoustic_kernel.cuh)
 * or TTI (warps per CTA, z unrolling, rows per thread; tti_kernel.cuh):
 * acoustic 0..12, TTI 0..12 (9..12, two rows per thread, up to order 8),
 * or -1 for the default of the solver's equation, order and storage.
 * Resets zchunks to its default.
 * fdw_get_tile_config returns the configuration in use (-1 for NULL).
 * Errors: INVALID_ARG.
 */
int fdw_set_tile_config(fdw_solver *s, int tile);
int fdw_get_tile_config(const fdw_solver *s);
int fdw_get_zchunks(const fdw_solver *s);

/*
 * ---- Adjoint and FWI gradient (acoustic) ----------------------------------
 * The paper motivates the solvers by FWI/RTM (Introduction) but states no
 * adjoint; these calls give the exact transpose of the discrete recurrence
 * above. For a residual res [(nt+1)][nrec] (dJ/d traces) the multipliers
 * mu_k (k = nt .. 1, mu_{nt+1} = mu_{nt+2} = 0) obey the same step run
 * backwards:  P mu_k = 2 mu_{k+1} - Q mu_{k+2} + c (lap mu_{k+1} + R^T res_k),
 * R^T spreading each residual with the trilinear weights (no 1/h^3). Then
 *   dJ/d wavelet[n][s] = sum_corner (w / h^3) mu_{n+1}   (source side),
 *   dJ/dm = -(1/dt^2) sum_n mu_{n+1} (P u_{n+1} - 2 u_n + Q u_{n-1})
 * with m = 1/v^2 the squared slowness (the sponge damping is held fixed).
 */

/*
 * Keep forward levels for the gradient: allocates a ring of nlevels (>= 3)
 * wavefield buffers (reused across calls), stores the two current levels,
 * and from now on every fdw_step stores the level it produces (level l goes
 * to slot l mod nlevels). A checkpointed gradient restores a segment's start
 * with fdw_set_wavefield / fdw_set_current_step, calls fdw_history_begin,
 * replays the segment with fdw_step, then runs the adjoint steps of that
 * segment. Errors: INVALID_ARG (TTI, nlevels < 3), OOM.
 */
int fdw_history_begin(fdw_solver *s, int nlevels);
int fdw_history_end(fdw_solver *s);

/*
 * Start an adjoint run: copies the residual [(nt+1)][nrec] FP64 (host or
 * device), zeroes the multipliers (level k = nt+1) and, when
 * accumulate_gradient is non-zero, the gradient accumulator. Allocates the
 * adjoint buffers on first use. Errors: STATE (no dt), INVALID_ARG, OOM.
 */
int fdw_adjoint_begin(fdw_solver *s, const double *residual, int nt, int ptr_is_device,
                      int accumulate_gradient);

/*
 * Advance the adjoint nsteps levels (k -> k - nsteps, nsteps <= k - 1): the
 * acoustic stencil kernel on the multiplier buffers, the residual spread,
 * the source-side adjoint, and (if accumulating) the gradient term of each
 * produced level, which needs forward levels j, j-1, j-2 in the history
 * (FDW_ERR_STATE otherwise). Asynchronous on the stream.
 */
int fdw_adjoint_step(fdw_solver *s, int nsteps);

/* Current adjoint level k (the multipliers hold mu_k, mu_{k+1}); -1 if none. */
int fdw_adjoint_current_step(const fdw_solver *s);

/*
 * dJ/dm on the PHYSICAL grid [nz][ny][nx] FP64 (host or device), m = 1/v^2:
 * the accumulated sum scaled by -1/dt^2, with the contributions of sponge
 * points added to the physical point whose medium they copy.
 * Errors: STATE (no gradient accumulated).
 */
int fdw_get_gradient(fdw_solver *s, double *grad_m, int ptr_is_device);

/*
 * Velocity gradient from the slowness-squared gradient (m = 1/v^2, so
 * dJ/dv = -2 v^-3 dJ/dm), elementwise over n points: vp FP32 m/s, grad_m
 * and grad_v FP64, all in device memory (grad_v may alias grad_m);
 * asynchronous on `stream`. Used by the FWI gradient after the per-shot
 * dJ/dm of fdw_get_gradient have been summed.
 * Errors: INVALID_ARG (NULL pointers with n > 0, n < 0), CUDA.
 */
int fdw_velocity_gradient(const float *vp, const double *grad_m, long long n, double *grad_v, void *stream);

/* dJ/d wavelet [nt][nsrc] FP64 of the adjoint run so far (host or device). */
int fdw_get_source_adjoint(fdw_solver *s, double *out, int ptr_is_device);

/*
 * FWI data misfit of traces d against observations d_obs (both n FP64
 * values in device memory): residual[i] = d[i] - d_obs[i] (skipped when
 * residual is NULL; it is the residual fdw_adjoint_begin takes) and
 * *J = 1/2 sum residual^2 (FP64, device memory). Deterministic: the sum is
 * taken over fixed chunks of 2048 values, then over the chunk sums in a
 * fixed order. Asynchronous on `stream` (a cudaStream_t or NULL); the chunk
 * sums live in a scratch buffer taken from the stream-ordered allocator
 * (cudaMallocAsync) and returned at the end of the call.
 * d and d_obs may be NULL when n = 0 (then *J = 0).
 * Errors: INVALID_ARG (NULL pointers, n < 0), OOM, CUDA.
 */
int fdw_misfit(const double *d, const double *d_obs, long long n, double *residual, double *J,
               void *stream);

/*
 * fdw_misfit without any device allocation. The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * themselves or have the library do it -- code that owns every byte of the
 * GPU through its own pool allocator, a real-time loop that cannot afford
 * the implicit synchronisation of cudaMalloc / cudaFree, or a process close
 * to running out of device memory.
 * Same arguments, results and determinism as fdw_misfit (the caller still
 * passes the inputs d, d_obs and the outputs residual, J in device memory),
 * but the chunk sums go to a scratch array compiled into the library: 256 KB
 * per GPU, held from the first use until the process exits. Limit:
 * n <= 67,108,864 values (32,768 chunks of 2048); larger n returns
 * FDW_ERR_INVALID_ARG with a message naming the limit.
 * The first call on a device looks up the scratch array's device address
 * (with that device current); make that first call before capturing the
 * stream into a CUDA graph. Every call, from any stream or thread, shares
 * the one scratch array of the device: calls that overlap on the GPU race
 * and must be serialised by the caller (e.g. issue them on one stream).
 * Nothing in the scratch needs clearing between calls (every chunk sum a
 * call reads, that call writes first). The looked-up address is kept for
 * the life of the process: do not use this entry point on a device after
 * cudaDeviceReset of that device (the module may be loaded again at
 * another address).
 * Errors: INVALID_ARG (NULL pointers, n < 0, n above the limit), CUDA.
 */
int fdw_misfit_noalloc(const double *d, const double *d_obs, long long n, double *residual,
                       double *J, void *stream);

/* Multipliers mu_k (level 0) or mu_{k+1} (level 1), layout of fdw_get_wavefield. */
int fdw_get_adjoint_wavefield(const fdw_solver *s, int level, float *out, int ptr_is_device);

/*
 * ---- Learned closure ------------------------------------------------------
 * The paper trades grid spacing against stencil order (Section "Cost-benefit
 * analysis"); it has no learned part. The closure is a 3x3x3 convolutional
 * network, 3 -> 16 -> 16 -> 1 channels with ReLU between, that corrects a
 * coarse low-order time step toward a fine high-order one:
 *   x = (u_n / s, u_{n-1} / s, (v - 3000 m/s) / 750 m/s),  s = max |u_n|
 *   over the computational grid (1e-30 if the level is zero),
 *   x0 = (0, 0, (v - 3000 m/s) / 750 m/s),
 *   u_{n+1} += s * (net(x) - net(x0))   (applied every coarse step, on the
 *   physical points 3 or more points away from the sponge, so that the
 *   7^3 receptive field is physical; elsewhere the plain update stands).
 * The correction vanishes wherever u_n and u_{n-1} vanish over the 7^3
 * receptive field: an output there would be integrated twice by the
 * leapfrog update and grow quadratically in time.
 * The velocity channel is the physical model extended by edge values into
 * the sponge, zero-padded outside the computational grid like u.
 * Parameters (fdw_closure_num_params() = 8673 FP32 values, BF16 copies of
 * the convolution weights used by the kernels, FP32 biases and
 * accumulation), concatenated:
 *   W1[16][3][27], b1[16], W2[16][16][27], b2[16], W3[1][16][27], b3[1],
 * tap t = (a*3 + b)*3 + c for the offsets (a-1, b-1, c-1) along (z, y, x)
 * (cross-correlation). Training works on batches of cubic patches
 * [batch][3][S][S][S] (FP32, device) with valid convolutions: the
 * correction net(x) - net(x0) is [batch][S-6][S-6][S-6]. Calls are ordered
 * on the closure's stream.
 */
typedef struct fdw_closure fdw_closure;

long long fdw_closure_num_params(void);

/* Create a closure with zero parameters on the current device. */
int fdw_closure_create(fdw_closure **out, void *stream);
int fdw_closure_destroy(fdw_closure *c);

/*
 * Inference kernels of fdw_step_closure: 0 (default) = one persistent kernel
 * on the Blackwell tensor cores (tcgen05.mma from shared memory into tensor
 * memory), 2 = one fused kernel on warp-level tensor-core MMAs (mma.sync);
 * both take FP16 operands (the BF16 weights exactly, the activations
 * rounded to FP16) with FP32 accumulation; 1 = plain FP32 convolutions on
 * the CUDA cores (the cross-check). Errors: INVALID_ARG.
 */
int fdw_closure_set_variant(fdw_closure *c, int variant);

/* Set (resets the Adam state) / read the FP32 parameters (host or device). */
int fdw_closure_set_params(fdw_closure *c, const float *params, int ptr_is_device);
int fdw_closure_get_params(fdw_closure *c, float *params, int ptr_is_device);

/* Correction net(x) - net(x0) of a patch batch: out [batch][S-6]^3 (device). */
int fdw_closure_forward(fdw_closure *c, const float *x, int batch, int S, float *out);

/*
 * Mean-squared error of the correction against target [batch][S-6]^3
 * (device), written to
 * *loss (device float), and its gradient w.r.t. the parameters into grad
 * (device, fdw_closure_num_params() floats; NULL for the loss only).
 * Deterministic: fixed-order reductions, no atomics.
 */
int fdw_closure_loss_grad(fdw_closure *c, const float *x, const float *target, int batch, int S,
                          float *loss, float *grad);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the batch's loss. */
int fdw_closure_adam_step(fdw_closure *c, const float *x, const float *target, int batch, int S,
                          float lr, float *loss);

/*
 * Advance the solver nsteps steps with the closure applied after each
 * stencil update (acoustic only; the closure and the solver must live on
 * the same device and their calls are ordered on the solver's stream).
 * Allocates the closure's inference workspace for the solver's grid on
 * first use. Errors: INVALID_ARG, STATE (no dt), OOM, CUDA.
 */
int fdw_step_closure(fdw_solver *s, fdw_closure *c, int nsteps);

/*
 * fdw_step_closure with the correction applied only on every `every`-th
 * step (the steps whose solver step count n, fdw_current_step before the
 * step, is a multiple of `every`; the others are plain steps) and
 * multiplied by `every` there, so that the correction per unit of time
 * stays the same at 1/every of the network's cost. The phase follows the
 * solver's step count, not the call: two calls of m steps correct the same
 * steps as one call of 2m. every = 1 is fdw_step_closure. Errors: as
 * fdw_step_closure; INVALID_ARG for every < 1.
 */
int fdw_step_closure_every(fdw_solver *s, fdw_closure *c, int nsteps, int every);

/*
 * Kernel timing. After fdw_profile_begin, up to max_launches (<= 65536)
 * stencil launches issued by fdw_step are bracketed by CUDA events recorded
 * on the solver's stream (steps are then launched individually instead of
 * as CUDA graphs). fdw_profile_end synchronises the stream and returns the
 * summed device time of those launches in milliseconds and their count.
 * Errors: INVALID_ARG, STATE (end without begin), CUDA.
 */
int fdw_profile_begin(fdw_solver *s, int max_launches);
int fdw_profile_end(fdw_solver *s, double *stencil_ms, int *launches);

#ifdef __cplusplus
}
#endif
#endif /* FDWAVE_H */
