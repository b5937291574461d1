// fdw_internal.h -- types shared by the translation units of libfdwave
// (sm_103a). Not part of the public C ABI (include/fdwave.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace fdw {

constexpr int kMaxR = 8;          // space order 16
constexpr int kTileX = 32;        // x extent of a stencil tile (one warp)
constexpr int kMaxZChunk = 256;  // most z planes one CTA of a 2.5D kernel marches

// Device error flags (bit mask written with atomicOr).
constexpr int kErrWaitTimeout = 1;  // an mbarrier wait gave up
constexpr int kErrBadLaunch = 2;    // a kernel saw inconsistent launch arguments

// Padded storage of one computational-grid field: x rows of Xp elements
// (Xp a multiple of 32, so every tile row is a full 128-byte line in FP32),
// NY rows per plane, NZ planes. Elements x in [NX, Xp) are padding and read
// as zero through the tensor maps (their extent is NX).
struct Dims {
  int NX, NY, NZ;
  int Xp;
  __host__ __device__ size_t plane() const { return (size_t)Xp * (size_t)NY; }
  __host__ __device__ size_t vol() const { return plane() * (size_t)NZ; }
};

// Central finite-difference weights at unit spacing, offsets 0..r.
struct Weights {
  float w2[kMaxR + 1];    // second derivative
  float c1[kMaxR + 1];    // first derivative (c1[0] = 0)
  float2 w2p[kMaxR + 1];  // w2 as pairs {w2, w2}, for packed FP32 arithmetic
  float2 c1p[kMaxR + 1];  // c1 as pairs {c1, c1}
  float2 c1n[kMaxR + 1];  // -c1 as pairs
};

// Damping tables: gh_a[i] = gamma_a(i) * dt / 2 for each axis.
struct Sponge {
  const float *gx, *gy, *gz;
};

// Storage-type traits: FP32 arithmetic on every storage type.
template <typename T> struct St;
template <> struct St<float> {
  static __device__ __forceinline__ float ld(float v) { return v; }
  static __device__ __forceinline__ float st(float v) { return v; }
  static constexpr CUtensorMapDataType tma = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
};
template <> struct St<__nv_bfloat16> {
  static __device__ __forceinline__ float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
  static constexpr CUtensorMapDataType tma = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
};
template <> struct St<__half> {
  static __device__ __forceinline__ float ld(__half v) { return __half2float(v); }
  static __device__ __forceinline__ __half st(float v) { return __float2half_rn(v); }
  static constexpr CUtensorMapDataType tma = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
};

// Host-side launchers (defined in the kernel translation units). Each
// returns a cudaError_t of the launch.

// Acoustic step (Eq. Acou + sponge): reads cur (level n), prev (n-1) and
// coefficient c (= (v dt / h)^2), writes level n+1 into prev's storage.
struct AcousticLaunch {
  int storage;            // FDW_F32 / FDW_BF16 / FDW_F16
  int r;                  // stencil radius (order / 2)
  Dims d;
  Weights w;
  Sponge sp;
  void *cur, *prev;       // fields (element type = storage)
  void *out;              // buffer of level n+1 (null: prev's storage, in place)
  const void *c;          // coefficient (storage type)
  const CUtensorMap *map_cur_halo, *map_cur_int, *map_prev_int, *map_c_int;
  int zchunks;            // CTAs along z
  int *err;               // device error flags
  int naive;              // 1 = one-thread-per-point kernel (debug cross-check)
  int prepare_only;       // 1 = only set kernel attributes (outside graph capture)
  int tile;               // tile configuration index of the 2.5D kernel
  int *occupancy_out;     // with prepare_only: resident CTAs per SM of the configuration
};
cudaError_t launch_acoustic(const AcousticLaunch &L, cudaStream_t st);
cudaError_t acoustic_prepare(int storage, int r, int tile);
// Resident CTAs per SM of a configuration (sets its attributes); 0 on error.
int acoustic_ctas_per_sm(int storage, int r, int tile);
int tti_ctas_per_sm(int storage, int r, int tile);

// Tile geometry of one configuration of the 2.5D acoustic kernel: the TMA
// boxes (halo tile and interior tiles) the host encodes in tensor maps.
struct TileGeom {
  int box_halo_x, box_halo_y, box_int_x, box_int_y, smem;
};
constexpr int kGraphSteps = 16;  // steps per CUDA graph of a long fdw_step run (even)
constexpr int kAcTiles = 13;  // number of configurations (see acoustic_kernel.cuh)
// 0 on success, -1 for an unknown (storage, r, tile).
int acoustic_geom(int storage, int r, int tile, TileGeom *g);
// Default configuration for (storage, r).
int acoustic_default_tile(int storage, int r);
cudaError_t launch_acoustic_f32(const AcousticLaunch &L, cudaStream_t st);
cudaError_t launch_acoustic_bf16(const AcousticLaunch &L, cudaStream_t st);
cudaError_t launch_acoustic_f16(const AcousticLaunch &L, cudaStream_t st);
int acoustic_geom_f32(int r, int tile, TileGeom *g);
int acoustic_geom_bf16(int r, int tile, TileGeom *g);
int acoustic_geom_f16(int r, int tile, TileGeom *g);

// TTI step (Eq. TTI / Eq. DiffOp + sponge).
struct TTILaunch {
  int storage;
  int r;
  Dims d;
  Weights w;
  Sponge sp;
  void *p_cur, *p_prev, *r_cur, *r_prev;
  const void *c;      // (v dt / h)^2
  const void *e;      // 1 + 2 eps
  const void *dl;     // sqrt(1 + 2 delta)
  const void *ax, *ay;  // symmetry axis x/y components (sin t cos f, sin t sin f); the
                        // z component is sqrt(1 - ax^2 - ay^2) (the operator depends on
                        // n n^T only, so the sign of n is free)
  int zchunks;
  int *err;
  int naive;
  int prepare_only;
  int tile;           // configuration index of the 2.5D kernel (tti_kernel.cuh)
  int *occupancy_out; // with prepare_only: resident CTAs per SM of the configuration
  // tensor maps: halo tiles of p, r at level n; interior tiles of p, r at
  // level n-1 and of the medium fields
  const CUtensorMap *m_ph, *m_rh, *m_pm, *m_rm, *m_c, *m_e, *m_d, *m_ax, *m_ay;
};
constexpr int kTtiTilesMax = 13;  // number of TTI configurations (see tti_kernel.cuh)
cudaError_t launch_tti(const TTILaunch &L, cudaStream_t st);
cudaError_t tti_prepare(int storage, int r, int tile);
int tti_geom(int storage, int r, int tile, TileGeom *g);
int tti_default_tile(int storage, int r);
cudaError_t launch_tti_tma_f32(const TTILaunch &L, cudaStream_t st);
cudaError_t launch_tti_tma_bf16(const TTILaunch &L, cudaStream_t st);
cudaError_t launch_tti_tma_f16(const TTILaunch &L, cudaStream_t st);
int tti_geom_f32(int r, int tile, TileGeom *g);
int tti_geom_bf16(int r, int tile, TileGeom *g);
int tti_geom_f16(int r, int tile, TileGeom *g);

// Sparse work of one step (after the stencil update):
//   inject: u+ += c w_corner amp / (h P) at each source corner (both p and r
//   for TTI); advances the device step counter.
//   gather: trace[n+1][rec] = sum_corner w u+(corner) in FP64.
struct SparseLaunch {
  int storage;
  Dims d;
  Sponge sp;
  void *f0, *f1;             // field(s) at the new level (f1 = r for TTI or null)
  const void *c;
  int nsrc;
  const int *src_corner;     // [nsrc*8*3] computational (i, j, k) of each corner
  const float *src_w;        // [nsrc*8] trilinear weight / h, 0 for dropped corners
  const float *wavelet;      // [nt_src][nsrc]
  int nt_src;
  int nrec;
  const int *rec_corner;
  const float *rec_w;
  double *traces;            // [(nt_rec+1)][nrec]
  int nt_rec;
  int *step;                 // device step counter n (of the level before the update)
  // adjoint mode: the residual row of the level being produced is spread
  // with receiver weights (no 1/h) -- see adjoint entry points
  const double *residual;    // [(nt_res+1)][nrec] or null
  int nt_res;
  float res_scale;           // h^2: c' = c / h^2 is stored, the adjoint source is c R^T res
  int adjoint;
  double *src_adj;           // [nt_src][nsrc] adjoint w.r.t. the wavelet, or null
  float src_adj_scale;       // 1 / (h^2 S)
  float amp_scale;           // S: stored fields are S x the physical ones
  double trace_scale;        // 1 / S
};
cudaError_t launch_sparse(const SparseLaunch &L, cudaStream_t st);

// Set the thread-local message of fdw_last_error and return `code`.
int report_error(int code, const char *fmt, ...);

// Learned closure (closure.cu): parameters and workspaces.
struct ClosureNet {
  cudaStream_t stream = nullptr;
  float *pf = nullptr;            // FP32 master parameters
  __nv_bfloat16 *pb = nullptr;    // BF16 copy used by the kernels
  float *grad = nullptr, *m = nullptr, *v = nullptr;  // gradient, Adam moments
  int adam_t = 0;
  // training workspace
  float *a1 = nullptr, *a2 = nullptr, *out = nullptr, *g3 = nullptr, *g2 = nullptr, *g1 = nullptr;
  float *partial = nullptr, *loss_partial = nullptr;
  // capacity (points per channel) of the layer-1/2/3 outputs of the workspace
  size_t cap1 = 0, cap2 = 0, cap3 = 0;
  float *xpair = nullptr;         // a batch and its zero-wavefield copy
  size_t xcap = 0;                // floats in xpair
  // inference workspace (one computational grid); base = net(0, 0, v)
  float *x = nullptr, *ia1 = nullptr, *ia2 = nullptr, *base = nullptr, *s_dev = nullptr;
  // tensor-core inference (closure_tc.cu, closure_umma.cu): FP16 inputs,
  // network output, operands of the mma.sync and tcgen05 kernels
  void *x16 = nullptr, *tcw = nullptr, *umw = nullptr;
  float *tc_out = nullptr;
  size_t tc_cap = 0;
  // 0: tcgen05 kernel (closure_umma.cu), 1: FP32 CUDA-core kernels,
  // 2: mma.sync kernel (closure_tc.cu)
  int variant = 0;
  float *s_partial = nullptr;     // per-block maxima of |u_n|
  size_t infer_cap = 0;           // points
};
// Once per fdw_step_closure call: base = net(0, 0, v) on the grid. `err`
// receives device-side wait timeouts (tcgen05 kernel).
cudaError_t closure_infer_base(ClosureNet *c, const float *vp, int nx, int ny, int nz, int nb, Dims d,
                               int *err, cudaStream_t st);
// Before the stencil of a step: s = max |u_n|, inputs, the first two layers.
cudaError_t closure_infer_pre(ClosureNet *c, int storage, const void *u, const void *um,
                              const float *vp, int nx, int ny, int nz, int nb, Dims d, int *err,
                              cudaStream_t st);
// After the stencil: u_{n+1} += factor * s * (last layer - base) on the
// physical points (sponge width nb, physical extents nx, ny, nz).
cudaError_t closure_infer_apply(ClosureNet *c, int storage, void *unew, Dims d, int nx, int ny, int nz, int nb,
                                float factor, cudaStream_t st);
int closure_reserve_infer(ClosureNet *c, Dims d);
// tensor-core path (closure_tc.cu)
int closure_tc_reserve(ClosureNet *c, Dims d);
cudaError_t closure_tc_base(ClosureNet *c, const float *vp, int nx, int ny, int nz, int nb, Dims d,
                            int *err, cudaStream_t st);
cudaError_t closure_tc_net(ClosureNet *c, int storage, const void *u, const void *um, const float *vp, int nx,
                           int ny, int nz, int nb, Dims d, int *err, cudaStream_t st);
// tcgen05 path (closure_umma.cu): operand buffer, operand preparation, the
// network on the FP16 inputs x16 into dst (FP32, dense [NZ][NY][NX])
int closure_umma_reserve(ClosureNet *c);
cudaError_t closure_umma_prepare(ClosureNet *c, cudaStream_t st);
// Points whose network output the time loop uses: those at least
// kClosureHalo points (the receptive-field radius of the three 3x3x3
// layers) inside the physical grid; [lo, hi) per axis (x, y, z) on the
// computational grid. The tensor-core kernels compute the output there
// only (the points of a work item beyond hi are computed and unused).
constexpr int kClosureHalo = 3;
struct NetBox {
  int lo[3], hi[3];
  bool empty() const { return hi[0] <= lo[0] || hi[1] <= lo[1] || hi[2] <= lo[2]; }
};
cudaError_t closure_umma_run(ClosureNet *c, const void *x16, float *dst, Dims d, const NetBox &box, int *err,
                             cudaStream_t st);

}  // namespace fdw

// The public closure handle of include/fdwave.h.
struct fdw_closure : fdw::ClosureNet {};

namespace fdw {

// FWI gradient kernels (adjoint.cu)
cudaError_t launch_grad_accum(int storage, const void *mu, const void *u1, const void *u0,
                              const void *um1, float *g32, Dims d, Sponge sp, cudaStream_t st);
// Terms j-1 and j-2 in one pass: mu_a = mu_j, mu_b = mu_{j-1}, ua..ud =
// u_j, u_{j-1}, u_{j-2}, u_{j-3} (ud may be null: u_{j-3} = 0).
cudaError_t launch_grad_accum_pair(int storage, const void *mu_a, const void *mu_b, const void *ua,
                                   const void *ub, const void *uc, const void *ud, float *g32, Dims d, Sponge sp,
                                   cudaStream_t st);
cudaError_t launch_grad_flush(float *g32, double *g64, size_t n, cudaStream_t st);
cudaError_t launch_grad_physical(const double *g64, Dims d, int nx, int ny, int nz, int nb,
                                 double scale, double *out, cudaStream_t st);

// Utility kernels (setup.cu)
cudaError_t launch_coef_acoustic(int storage, const float *vp_phys, int nx, int ny, int nz,
                                 int nb, Dims d, double dt_over_h, void *c, cudaStream_t st);
cudaError_t launch_coef_tti(int storage, const float *vp, const float *eps, const float *delta,
                            const float *theta, const float *phi, int nx, int ny, int nz,
                            int nb, Dims d, double dt_over_h, void *c, void *e, void *dl,
                            void *ax, void *ay, cudaStream_t st);
cudaError_t launch_max_velocity(const float *vp, const float *eps, const float *theta, long n, float *out4,
                                cudaStream_t st);
// dense [NZ][NY][NX] f32 <-> padded storage, values multiplied by `scale`
cudaError_t launch_pack(int storage, const float *src, void *dst, Dims d, float scale,
                        cudaStream_t st);
cudaError_t launch_unpack(int storage, const void *src, Dims d, float *dst, float scale,
                          cudaStream_t st);
cudaError_t launch_nonfinite(int storage, const void *f, Dims d, int *flag, cudaStream_t st);

}  // namespace fdw
