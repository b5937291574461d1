// fdw_api.cu -- the C ABI declared in include/fdwave.h: solver lifetime,
// medium/dt/sparse-point set-up and the CUDA-graph time loop of Algorithm 1.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "fdw_internal.h"
#include "fdwave.h"

using namespace fdw;

// --------------------------------------------------------------------------
// errors
// --------------------------------------------------------------------------
static thread_local char g_err[1024];

static int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

// Error reporting for the other translation units of the library.
int fdw::report_error(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

static int cuda_fail(cudaError_t e, const char *what) {
  cudaGetLastError();  // clear a non-sticky error
  return fail(e == cudaErrorMemoryAllocation ? FDW_ERR_OOM : FDW_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CK(x)                                         \
  do {                                                \
    cudaError_t e_ = (x);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x);  \
  } while (0)

extern "C" const char *fdw_last_error(void) { return g_err; }
extern "C" const char *fdw_version(void) { return "fdwave 0.1 (sm_103a)"; }

// --------------------------------------------------------------------------
// solver
// --------------------------------------------------------------------------
struct fdw_solver {
  int nx, ny, nz, nb, eq, order, r, storage, el;
  double h;
  Dims d;
  int device;
  cudaStream_t stream;  // caller's stream (may be NULL)
  cudaStream_t cap;     // private stream used only to capture graphs

  void *f[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [field][buffer]
  int cur = 0;          // buffer holding level n

  void *c = nullptr, *e = nullptr, *dl = nullptr, *ax = nullptr, *ay = nullptr;
  float *vp = nullptr, *eps = nullptr, *delta = nullptr, *theta = nullptr, *phi = nullptr;
  float *gam[3] = {nullptr, nullptr, nullptr};
  float *scratch2 = nullptr;  // 4 words: model maxima / flags
  bool model_set = false, dt_set = false;
  double vmax = 0, vmax_eff = 0, dt = 0;
  double sponge_vref = 0.0, sponge_R = 1e-3;  // vref <= 0: the model's vmax
  // stored wavefields are fscale x the physical ones (keeps FP16 storage in
  // its normal range); fscale_req = 0 means automatic
  double fscale = 1.0, fscale_req = 0.0;

  int nsrc = 0, nt_src = 0;
  int *src_corner = nullptr;
  float *src_w = nullptr, *wavelet = nullptr;
  int nrec = 0, nt_rec = 0;
  int *rec_corner = nullptr;
  float *rec_w = nullptr;
  double *traces = nullptr;

  int *d_step = nullptr, *d_err = nullptr;
  int it = 0;

  Weights w;
  int zchunks = 0;
  int tile = 0;  // configuration of the 2.5D acoustic kernel
  int naive = 0;
  CUtensorMap map_halo[2][2], map_int[2][2], map_c;  // [field][buffer]
  CUtensorMap map_e, map_dl, map_ax, map_ay;          // TTI medium
  bool maps_ok = false;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};      // one step, per buffer parity
  cudaGraphExec_t graph_run[2] = {nullptr, nullptr};  // kGraphSteps steps, per parity
  bool graph_ok = false;

  // profiling: CUDA events around each stencil launch (direct launches)
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  int prof_n = 0;

  // adjoint (acoustic): multipliers mu_k in a[acur], mu_{k+1} in a[1-acur]
  void *a[2] = {nullptr, nullptr};
  int acur = 0;
  CUtensorMap amap_halo[2], amap_int[2];
  bool amaps_ok = false;
  bool adj_on = false, adj_grad = false;
  int ak = 0;                       // current adjoint level k
  double *residual = nullptr;       // [(nt_res+1)][nrec]
  int nt_res = 0;
  size_t residual_cap = 0;
  double *src_adj = nullptr;        // [nt_src][nsrc]
  int *d_astep = nullptr;
  float *grad32 = nullptr;          // FP32 partial sums of the current segment
  double *grad64 = nullptr;         // FP64 total (computational grid, unscaled)
  int grad_pending = 0;             // terms in grad32 not yet flushed

  // forward history ring (levels of u for the gradient)
  std::vector<void *> hist;
  std::vector<int> hist_level;
  std::vector<CUtensorMap> hmap_halo, hmap_int;  // tensor maps of the ring buffers
  bool hist_on = false;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

// Central weights at unit spacing, closed forms (order 2r):
//   second derivative: w_j = 2 (-1)^(j+1) (r!)^2 / (j^2 (r-j)! (r+j)!), w_0 = -2 sum w_j
//   first derivative:  c_j =   (-1)^(j+1) (r!)^2 / (j   (r-j)! (r+j)!)
void closed_form_weights(int r, double *w2, double *c1) {
  double s = 0.0;
  for (int j = 1; j <= r; ++j) {
    double ratio = 1.0;  // (r!)^2 / ((r-j)! (r+j)!)
    for (int i = 0; i < j; ++i) ratio *= (double)(r - i) / (double)(r + i + 1);
    const double sg = (j % 2 == 1) ? 1.0 : -1.0;
    w2[j] = 2.0 * sg * ratio / ((double)j * j);
    c1[j] = sg * ratio / (double)j;
    s += w2[j];
  }
  w2[0] = -2.0 * s;
  c1[0] = 0.0;
}

// Sum of |weights| of the 3D Laplacian stencil (a2 of Eq. stability).
double laplacian_a2(int r) {
  double w2[kMaxR + 1], c1[kMaxR + 1];
  closed_form_weights(r, w2, c1);
  double s = fabs(w2[0]);
  for (int j = 1; j <= r; ++j) s += 2.0 * fabs(w2[j]);
  return 3.0 * s;
}

template <typename P>
cudaError_t dmalloc(P **p, size_t bytes) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  *p = (P *)q;
  return e;
}

void dfree(void *p) {
  if (p) cudaFree(p);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

CUtensorMapDataType tma_type(int storage) {
  return storage == FDW_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
         : storage == FDW_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
}

int make_map(CUtensorMap *m, const fdw_solver *s, void *base, int bx, int by) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return fail(FDW_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const cuuint64_t dims[3] = {(cuuint64_t)s->d.NX, (cuuint64_t)s->d.NY, (cuuint64_t)s->d.NZ};
  const cuuint64_t strides[2] = {(cuuint64_t)s->d.Xp * s->el, (cuuint64_t)s->d.plane() * s->el};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, tma_type(s->storage), 3, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(FDW_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return FDW_OK;
}

int build_maps(fdw_solver *s) {
  if (s->maps_ok) return FDW_OK;
  TileGeom tg;
  const int bad = s->eq == FDW_TTI ? tti_geom(s->storage, s->r, s->tile, &tg)
                                   : acoustic_geom(s->storage, s->r, s->tile, &tg);
  if (bad) return fail(FDW_ERR_INVALID_ARG, "bad tile");
  const int bhx = tg.box_halo_x, bhy = tg.box_halo_y, bix = tg.box_int_x, biy = tg.box_int_y;
  const int nf = s->eq == FDW_TTI ? 2 : 1;
  for (int f = 0; f < nf; ++f)
    for (int b = 0; b < 2; ++b) {
      int rc = make_map(&s->map_halo[f][b], s, s->f[f][b], bhx, bhy);
      if (rc) return rc;
      rc = make_map(&s->map_int[f][b], s, s->f[f][b], bix, biy);
      if (rc) return rc;
    }
  int rc = make_map(&s->map_c, s, s->c, bix, biy);
  if (rc) return rc;
  if (s->eq == FDW_TTI) {
    if ((rc = make_map(&s->map_e, s, s->e, bix, biy))) return rc;
    if ((rc = make_map(&s->map_dl, s, s->dl, bix, biy))) return rc;
    if ((rc = make_map(&s->map_ax, s, s->ax, bix, biy))) return rc;
    if ((rc = make_map(&s->map_ay, s, s->ay, bix, biy))) return rc;
  }
  s->maps_ok = true;
  return FDW_OK;
}

void drop_graphs(fdw_solver *s) {
  for (int b = 0; b < 2; ++b) {
    if (s->graph[b]) {
      cudaGraphExecDestroy(s->graph[b]);
      s->graph[b] = nullptr;
    }
    if (s->graph_run[b]) {
      cudaGraphExecDestroy(s->graph_run[b]);
      s->graph_run[b] = nullptr;
    }
  }
  s->graph_ok = false;
}

// A CTA marches at most kMaxZChunk planes (its damping slice lives in
// shared memory).
int min_zchunks(const fdw_solver *s) { return (s->d.NZ + kMaxZChunk - 1) / kMaxZChunk; }

// Default number of z chunks of the 2.5D kernels (measured on the 592^3
// acoustic and the 464^3 and 212^3 TTI workloads).
// FP32 acoustic and TTI kernels: a CTA marching a chunk of L planes does
// L + 2r plane iterations (the queue fill) and the grid runs in waves of
// (SMs x resident CTAs per SM); the time is modelled as
//   ceil(CTAs / slots) x (ceil(NZ / chunks) + 2r)
// and minimised over the chunk counts that keep at least max(4, r) planes
// per chunk: this picks the measured best chunking at every order of the
// 592^3 acoustic workload, ranks the TTI chunkings of the 212^3 grid as
// measured, and gives many short chunks on grids that fit in one wave.
// The 16-bit acoustic kernels (more resident CTAs, short fills) run best
// with more, smaller chunks: about 32 CTAs per SM in total.
int default_zchunks(const fdw_solver *s) {
  TileGeom tg;
  const bool tti = s->eq == FDW_TTI;
  const int bad = tti ? tti_geom(s->storage, s->r, s->tile, &tg) : acoustic_geom(s->storage, s->r, s->tile, &tg);
  if (bad) return 1;
  const long tiles = (long)((s->d.NX + tg.box_int_x - 1) / tg.box_int_x) * ((s->d.NY + tg.box_int_y - 1) / tg.box_int_y);
  // chunks of at least 4 planes (and r): on small grids that fit in one
  // wave, shorter chunks shorten every CTA's serial march
  const int zmin = s->r > 4 ? s->r : 4;
  long maxch = s->d.NZ / zmin;
  if (maxch < 1) maxch = 1;
  const int lo = min_zchunks(s);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 152;
  }
  if (!tti && s->storage != FDW_F32) {
    long want = ((long)sms * 32 + tiles - 1) / tiles;
    if (want > maxch) want = maxch;
    if (want < 1) want = 1;
    return lo > want ? lo : (int)want;
  }
  // FP32 acoustic and TTI: the chunk count that minimises waves x planes
  // marched per CTA (chunk length + the 2r halo planes)
  int occ = tti ? tti_ctas_per_sm(s->storage, s->r, s->tile) : acoustic_ctas_per_sm(s->storage, s->r, s->tile);
  if (occ < 1) occ = 1;
  const long slots = (long)sms * occ;
  long best = lo, best_cost = -1;
  for (long ch = lo; ch <= (maxch > lo ? maxch : lo); ++ch) {
    const long len = (s->d.NZ + ch - 1) / ch;
    const long used = (s->d.NZ + len - 1) / len;  // chunks actually launched
    const long waves = (tiles * used + slots - 1) / slots;
    const long cost = waves * (len + 2 * s->r);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = ch;
    }
  }
  return (int)best;
}

// Enqueue the stencil update of one time step from buffer `cur` on stream st.
int enqueue_stencil(fdw_solver *s, int cur, cudaStream_t st) {
  const int nxt = 1 - cur;
  if (s->eq == FDW_ACOUSTIC) {
    AcousticLaunch L{};
    L.storage = s->storage;
    L.r = s->r;
    L.d = s->d;
    L.w = s->w;
    L.sp = Sponge{s->gam[0], s->gam[1], s->gam[2]};
    L.cur = s->f[0][cur];
    L.prev = s->f[0][nxt];
    L.c = s->c;
    L.map_cur_halo = &s->map_halo[0][cur];
    L.map_cur_int = &s->map_int[0][cur];
    L.map_prev_int = &s->map_int[0][nxt];
    L.map_c_int = &s->map_c;
    L.zchunks = s->zchunks;
    L.err = s->d_err;
    L.naive = s->naive;
    L.tile = s->tile;
    CK(launch_acoustic(L, st));
  } else {
    TTILaunch L{};
    L.storage = s->storage;
    L.r = s->r;
    L.d = s->d;
    L.w = s->w;
    L.sp = Sponge{s->gam[0], s->gam[1], s->gam[2]};
    L.p_cur = s->f[0][cur];
    L.p_prev = s->f[0][nxt];
    L.r_cur = s->f[1][cur];
    L.r_prev = s->f[1][nxt];
    L.c = s->c;
    L.e = s->e;
    L.dl = s->dl;
    L.ax = s->ax;
    L.ay = s->ay;
    L.m_ph = &s->map_halo[0][cur];
    L.m_rh = &s->map_halo[1][cur];
    L.m_pm = &s->map_int[0][nxt];
    L.m_rm = &s->map_int[1][nxt];
    L.m_c = &s->map_c;
    L.m_e = &s->map_e;
    L.m_d = &s->map_dl;
    L.m_ax = &s->map_ax;
    L.m_ay = &s->map_ay;
    L.zchunks = s->zchunks;
    L.err = s->d_err;
    L.naive = s->naive;
    L.tile = s->tile;
    CK(launch_tti(L, st));
  }
  return FDW_OK;
}

// Enqueue the sparse work (injection, receivers) after the update from `cur`.
int enqueue_sparse(fdw_solver *s, int cur, cudaStream_t st) {
  const int nxt = 1 - cur;
  SparseLaunch S{};
  memset(&S, 0, sizeof S);
  S.storage = s->storage;
  S.d = s->d;
  S.sp = Sponge{s->gam[0], s->gam[1], s->gam[2]};
  S.f0 = s->f[0][nxt];
  S.f1 = s->eq == FDW_TTI ? s->f[1][nxt] : nullptr;
  S.c = s->c;
  S.nsrc = s->nsrc;
  S.src_corner = s->src_corner;
  S.src_w = s->src_w;
  S.wavelet = s->wavelet;
  S.amp_scale = (float)s->fscale;
  S.trace_scale = 1.0 / s->fscale;
  S.nt_src = s->nt_src;
  S.nrec = s->nrec;
  S.rec_corner = s->rec_corner;
  S.rec_w = s->rec_w;
  S.traces = s->traces;
  S.nt_rec = s->nt_rec;
  S.step = s->d_step;
  S.adjoint = 0;
  CK(launch_sparse(S, st));
  return FDW_OK;
}

int enqueue_step(fdw_solver *s, int cur, cudaStream_t st) {
  int rc = enqueue_stencil(s, cur, st);
  return rc ? rc : enqueue_sparse(s, cur, st);
}

int corners_of(const fdw_solver *s, int n, const double *xyz, double scale, std::vector<int> &ijk,
               std::vector<float> &wt) {
  ijk.assign((size_t)n * 24, 0);
  wt.assign((size_t)n * 8, 0.f);
  const int Ncomp[3] = {s->d.NX, s->d.NY, s->d.NZ};
  for (int p = 0; p < n; ++p) {
    int b[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
      const double v = xyz[3 * p + a];
      if (!isfinite(v)) return fail(FDW_ERR_OUT_OF_DOMAIN, "point %d: non-finite position", p);
      const double f = v / s->h + s->nb;
      if (f < 0.0 || f > (double)(Ncomp[a] - 1))
        return fail(FDW_ERR_OUT_OF_DOMAIN, "point %d axis %d: %g m is outside the grid", p, a, v);
      b[a] = (int)floor(f);
      t[a] = f - b[a];
    }
    for (int q = 0; q < 8; ++q) {
      int id[3];
      double wq = 1.0;
      bool inside = true;
      for (int a = 0; a < 3; ++a) {
        const int bit = (q >> a) & 1;
        id[a] = b[a] + bit;
        wq *= bit ? t[a] : 1.0 - t[a];
        if (id[a] > Ncomp[a] - 1) {
          inside = false;
          id[a] = Ncomp[a] - 1;
        }
      }
      for (int a = 0; a < 3; ++a) ijk[((size_t)p * 8 + q) * 3 + a] = id[a];
      wt[(size_t)p * 8 + q] = inside ? (float)(wq * scale) : 0.f;
    }
  }
  return FDW_OK;
}

int upload(void *dst, const void *src, size_t bytes, int is_dev, cudaStream_t st) {
  CK(cudaMemcpyAsync(dst, src, bytes, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  if (!is_dev) CK(cudaStreamSynchronize(st));
  return FDW_OK;
}

}  // namespace

// --------------------------------------------------------------------------
// lifetime
// --------------------------------------------------------------------------
extern "C" int fdw_destroy(fdw_solver *s) {
  if (!s) return FDW_OK;
  DeviceGuard g(s->device);
  cudaStreamSynchronize(s->stream);
  drop_graphs(s);
  for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
  for (int f = 0; f < 2; ++f)
    for (int b = 0; b < 2; ++b) dfree(s->f[f][b]);
  dfree(s->c); dfree(s->e); dfree(s->dl); dfree(s->ax); dfree(s->ay);
  dfree(s->vp); dfree(s->eps); dfree(s->delta); dfree(s->theta); dfree(s->phi);
  for (int a = 0; a < 3; ++a) dfree(s->gam[a]);
  dfree(s->scratch2);
  dfree(s->src_corner); dfree(s->src_w); dfree(s->wavelet);
  dfree(s->rec_corner); dfree(s->rec_w); dfree(s->traces);
  dfree(s->d_step); dfree(s->d_err);
  dfree(s->a[0]); dfree(s->a[1]); dfree(s->residual); dfree(s->src_adj); dfree(s->d_astep);
  dfree(s->grad32); dfree(s->grad64);
  for (void *p : s->hist) dfree(p);
  if (s->cap) cudaStreamDestroy(s->cap);
  delete s;
  return FDW_OK;
}

extern "C" int fdw_create(fdw_solver **out, int nx, int ny, int nz, double h, int nb, int equation,
                          int space_order, int storage, void *stream) {
  if (!out) return fail(FDW_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || nb < 0) return fail(FDW_ERR_INVALID_ARG, "bad grid size");
  if (!(h > 0.0) || !isfinite(h)) return fail(FDW_ERR_INVALID_ARG, "h must be positive");
  if (equation != FDW_ACOUSTIC && equation != FDW_TTI)
    return fail(FDW_ERR_INVALID_ARG, "unknown equation %d", equation);
  if (space_order < 2 || space_order > 2 * kMaxR || (space_order & 1))
    return fail(FDW_ERR_INVALID_ARG, "space order must be even in [2, %d]", 2 * kMaxR);
  if (storage != FDW_F32 && storage != FDW_BF16 && storage != FDW_F16)
    return fail(FDW_ERR_INVALID_ARG, "unknown storage %d", storage);
  const long NX = (long)nx + 2L * nb, NY = (long)ny + 2L * nb, NZ = (long)nz + 2L * nb;
  if (NX > (1L << 20) || NY > (1L << 20) || NZ > (1L << 20) || NX * NY > (1L << 31))
    return fail(FDW_ERR_INVALID_ARG, "grid too large");

  fdw_solver *s = new (std::nothrow) fdw_solver;
  if (!s) return fail(FDW_ERR_OOM, "host allocation failed");
  s->nx = nx; s->ny = ny; s->nz = nz; s->nb = nb; s->h = h;
  s->eq = equation; s->order = space_order; s->r = space_order / 2; s->storage = storage;
  s->el = storage == FDW_F32 ? 4 : 2;
  s->d.NX = (int)NX; s->d.NY = (int)NY; s->d.NZ = (int)NZ;
  s->d.Xp = (int)((NX + 31) / 32 * 32);
  s->stream = (cudaStream_t)stream;
  s->cap = nullptr;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return fail(FDW_ERR_CUDA, "no CUDA device");
  }
  {
    double w2[kMaxR + 1], c1[kMaxR + 1];
    closed_form_weights(s->r, w2, c1);
    for (int j = 0; j <= kMaxR; ++j) {
      s->w.w2[j] = j <= s->r ? (float)w2[j] : 0.f;
      s->w.c1[j] = j <= s->r ? (float)c1[j] : 0.f;
      s->w.w2p[j] = make_float2(s->w.w2[j], s->w.w2[j]);
      s->w.c1p[j] = make_float2(s->w.c1[j], s->w.c1[j]);
      s->w.c1n[j] = make_float2(-s->w.c1[j], -s->w.c1[j]);
    }
  }
  int rc = FDW_OK;
  auto try_alloc = [&](void **p, size_t bytes) {
    if (rc) return;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc");
  };
  const size_t fb = s->d.vol() * s->el;
  const int nf = equation == FDW_TTI ? 2 : 1;
  for (int f = 0; f < nf; ++f)
    for (int b = 0; b < 2; ++b) try_alloc(&s->f[f][b], fb);
  try_alloc(&s->c, fb);
  if (equation == FDW_TTI) {
    try_alloc(&s->e, fb); try_alloc(&s->dl, fb); try_alloc(&s->ax, fb); try_alloc(&s->ay, fb);
  }
  // the physical model's copies, filled by fdw_set_model (allocated here so
  // that setting a model allocates nothing)
  const size_t nphys = (size_t)nx * ny * nz * sizeof(float);
  try_alloc((void **)&s->vp, nphys);
  if (equation == FDW_TTI) {
    try_alloc((void **)&s->eps, nphys); try_alloc((void **)&s->delta, nphys);
    try_alloc((void **)&s->theta, nphys); try_alloc((void **)&s->phi, nphys);
  }
  try_alloc((void **)&s->gam[0], sizeof(float) * NX);
  try_alloc((void **)&s->gam[1], sizeof(float) * NY);
  try_alloc((void **)&s->gam[2], sizeof(float) * NZ);
  try_alloc((void **)&s->scratch2, 4 * sizeof(float));
  try_alloc((void **)&s->d_step, sizeof(int));
  try_alloc((void **)&s->d_err, sizeof(int));
  if (!rc && cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess)
    rc = fail(FDW_ERR_CUDA, "stream creation failed");
  if (!rc) {
    for (int f = 0; f < nf && !rc; ++f)
      for (int b = 0; b < 2 && !rc; ++b)
        if (cudaMemsetAsync(s->f[f][b], 0, fb, s->stream) != cudaSuccess) rc = fail(FDW_ERR_CUDA, "memset");
    if (!rc && (cudaMemsetAsync(s->c, 0, fb, s->stream) != cudaSuccess ||
                cudaMemsetAsync(s->d_step, 0, sizeof(int), s->stream) != cudaSuccess ||
                cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream) != cudaSuccess ||
                cudaStreamSynchronize(s->stream) != cudaSuccess))
      rc = fail(FDW_ERR_CUDA, "initialisation failed");
  }
  if (rc) {
    fdw_destroy(s);
    return rc;
  }
  s->tile = s->eq == FDW_TTI ? tti_default_tile(storage, s->r) : acoustic_default_tile(storage, s->r);
  s->zchunks = default_zchunks(s);
  const char *nv = getenv("FDW_KERNEL");
  s->naive = (nv && strcmp(nv, "naive") == 0) ? 1 : 0;
  *out = s;
  return FDW_OK;
}

// --------------------------------------------------------------------------
// medium, dt
// --------------------------------------------------------------------------
extern "C" int fdw_set_model(fdw_solver *s, const float *vp, const float *eps, const float *delta,
                             const float *theta, const float *phi, int ptr_is_device) {
  if (!s || !vp) return fail(FDW_ERR_INVALID_ARG, "NULL solver or vp");
  const bool tti = s->eq == FDW_TTI;
  if (tti && (!eps || !delta || !theta || !phi))
    return fail(FDW_ERR_INVALID_ARG, "TTI needs eps, delta, theta, phi");
  DeviceGuard g(s->device);
  const size_t n = (size_t)s->nx * s->ny * s->nz;
  auto ensure = [&](float **p) -> int {
    if (!*p) CK(dmalloc(p, n * sizeof(float)));
    return FDW_OK;
  };
  int rc = ensure(&s->vp);
  if (!rc && tti) rc = ensure(&s->eps);
  if (!rc && tti) rc = ensure(&s->delta);
  if (!rc && tti) rc = ensure(&s->theta);
  if (!rc && tti) rc = ensure(&s->phi);
  if (rc) return rc;
  const cudaMemcpyKind k = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(s->vp, vp, n * sizeof(float), k, s->stream));
  if (tti) {
    CK(cudaMemcpyAsync(s->eps, eps, n * sizeof(float), k, s->stream));
    CK(cudaMemcpyAsync(s->delta, delta, n * sizeof(float), k, s->stream));
    CK(cudaMemcpyAsync(s->theta, theta, n * sizeof(float), k, s->stream));
    CK(cudaMemcpyAsync(s->phi, phi, n * sizeof(float), k, s->stream));
  }
  CK(launch_max_velocity(s->vp, tti ? s->eps : nullptr, tti ? s->theta : nullptr, (long)n, s->scratch2,
                         s->stream));
  float vm[4];
  CK(cudaMemcpyAsync(vm, s->scratch2, sizeof vm, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  int bad;
  memcpy(&bad, &vm[2], sizeof bad);
  if (bad || !(vm[0] > 0.f) || !isfinite(vm[0]) || !isfinite(vm[1])) {
    s->model_set = false;
    s->dt_set = false;
    return fail(FDW_ERR_INVALID_ARG, "vp must be positive and finite everywhere (max %g)", (double)vm[0]);
  }
  // 16-bit storage keeps the axis as (nx, ny) and rebuilds nz = sqrt(1 -
  // nx^2 - ny^2): the rounding of nx, ny enters the cross coefficients
  // nx nz, ny nz amplified by about 1 / (2 nz), so beyond 75 degrees of tilt
  // (1 / (2 cos 75) ~ 2) the rebuilt axis is no longer at the storage's own
  // precision: such models need FP32 storage.
  if (tti && s->storage != FDW_F32 && vm[3] > 1.f - 0.258819045f) {
    s->model_set = false;
    s->dt_set = false;
    return fail(FDW_ERR_INVALID_ARG,
                "tilt up to %.1f degrees: 16-bit storage of the TTI axis is limited to 75 degrees "
                "(use FP32 storage)",
                acos(1.0 - (double)vm[3]) * 180.0 / M_PI);
  }
  s->vmax = vm[0];
  s->vmax_eff = vm[1];
  s->model_set = true;
  s->dt_set = false;
  drop_graphs(s);
  return FDW_OK;
}

extern "C" double fdw_max_stable_dt(const fdw_solver *s) {
  if (!s || !s->model_set) return -1.0;
  return s->h * sqrt(4.0 / laplacian_a2(s->r)) / s->vmax_eff;
}

extern "C" int fdw_set_dt(fdw_solver *s, double dt) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  if (!s->model_set) return fail(FDW_ERR_STATE, "fdw_set_model must come before fdw_set_dt");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(FDW_ERR_INVALID_ARG, "dt must be positive");
  const double dmax = fdw_max_stable_dt(s);
  if (dt > dmax * (1.0 + 1e-12))
    return fail(FDW_ERR_UNSTABLE_DT, "dt = %g exceeds the CFL limit %g (Eq. stability)", dt, dmax);
  DeviceGuard g(s->device);
  s->dt = dt;
  // sponge: gamma_a(i) = gamma_max d(i) / nb, gamma_max = 3 vmax ln(1/R) / (2 nb h), R = 1e-3,
  // d(i) = distance (in points) into the sponge; the tables hold gamma dt / 2.
  const double R = s->sponge_R;
  const double vref = s->sponge_vref > 0.0 ? s->sponge_vref : s->vmax;
  const double gmax = s->nb > 0 ? 3.0 * vref * log(1.0 / R) / (2.0 * s->nb * s->h) : 0.0;
  const int Ns[3] = {s->d.NX, s->d.NY, s->d.NZ};
  const int ns[3] = {s->nx, s->ny, s->nz};
  for (int a = 0; a < 3; ++a) {
    std::vector<float> t((size_t)Ns[a]);
    for (int i = 0; i < Ns[a]; ++i) {
      int dd = 0;
      if (i < s->nb) dd = s->nb - i;
      else if (i >= s->nb + ns[a]) dd = i - (s->nb + ns[a] - 1);
      t[i] = (float)(0.5 * dt * (s->nb > 0 ? gmax * dd / s->nb : 0.0));
    }
    CK(cudaMemcpyAsync(s->gam[a], t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  const double doh = dt / s->h;
  if (s->eq == FDW_ACOUSTIC) {
    CK(launch_coef_acoustic(s->storage, s->vp, s->nx, s->ny, s->nz, s->nb, s->d, doh, s->c, s->stream));
  } else {
    CK(launch_coef_tti(s->storage, s->vp, s->eps, s->delta, s->theta, s->phi, s->nx, s->ny, s->nz,
                       s->nb, s->d, doh, s->c, s->e, s->dl, s->ax, s->ay, s->stream));
  }
  // field scale: FP16 storage keeps the injected increment of a unit source
  // near 256 (a power of two, so scaling is exact); other storage types 1
  if (s->fscale_req > 0.0) {
    s->fscale = s->fscale_req;
  } else if (s->storage == FDW_F16) {
    const double cmax = (s->vmax_eff * dt / s->h) * (s->vmax_eff * dt / s->h);
    s->fscale = exp2(round(log2(256.0 * s->h / (cmax > 0.0 ? cmax : 1.0))));
  } else {
    s->fscale = 1.0;
  }
  s->dt_set = true;
  drop_graphs(s);
  return FDW_OK;
}

// --------------------------------------------------------------------------
// sources, receivers
// --------------------------------------------------------------------------
extern "C" int fdw_set_sources(fdw_solver *s, int nsrc, const double *xyz, const float *wavelet,
                               int nt, int ptr_is_device) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  if (nsrc < 0 || nt < 0) return fail(FDW_ERR_INVALID_ARG, "negative nsrc or nt");
  if (nsrc > 0 && (!xyz || (!wavelet && nt > 0))) return fail(FDW_ERR_INVALID_ARG, "NULL positions or wavelet");
  DeviceGuard g(s->device);
  std::vector<int> ijk;
  std::vector<float> wt;
  if (nsrc > 0) {
    int rc = corners_of(s, nsrc, xyz, 1.0 / s->h, ijk, wt);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(s->stream));
  dfree(s->src_corner); dfree(s->src_w); dfree(s->wavelet);
  s->src_corner = nullptr; s->src_w = nullptr; s->wavelet = nullptr;
  s->nsrc = 0; s->nt_src = 0;
  drop_graphs(s);
  if (nsrc == 0) return FDW_OK;
  CK(dmalloc(&s->src_corner, ijk.size() * sizeof(int)));
  CK(dmalloc(&s->src_w, wt.size() * sizeof(float)));
  CK(dmalloc(&s->wavelet, (size_t)(nt > 0 ? nt : 1) * nsrc * sizeof(float)));
  CK(cudaMemcpyAsync(s->src_corner, ijk.data(), ijk.size() * sizeof(int), cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(s->src_w, wt.data(), wt.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream));
  if (nt > 0) {
    int rc = upload(s->wavelet, wavelet, (size_t)nt * nsrc * sizeof(float), ptr_is_device, s->stream);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(s->stream));
  s->nsrc = nsrc;
  s->nt_src = nt;
  return FDW_OK;
}

extern "C" int fdw_set_receivers(fdw_solver *s, int nrec, const double *xyz, int nt) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  if (nrec < 0 || nt < 0) return fail(FDW_ERR_INVALID_ARG, "negative nrec or nt");
  if (nrec > 0 && !xyz) return fail(FDW_ERR_INVALID_ARG, "NULL receiver positions");
  DeviceGuard g(s->device);
  std::vector<int> ijk;
  std::vector<float> wt;
  if (nrec > 0) {
    int rc = corners_of(s, nrec, xyz, 1.0, ijk, wt);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(s->stream));
  dfree(s->rec_corner); dfree(s->rec_w); dfree(s->traces);
  s->rec_corner = nullptr; s->rec_w = nullptr; s->traces = nullptr;
  s->nrec = 0; s->nt_rec = 0;
  drop_graphs(s);
  if (nrec == 0) return FDW_OK;
  CK(dmalloc(&s->rec_corner, ijk.size() * sizeof(int)));
  CK(dmalloc(&s->rec_w, wt.size() * sizeof(float)));
  CK(dmalloc(&s->traces, (size_t)(nt + 1) * nrec * sizeof(double)));
  CK(cudaMemcpyAsync(s->rec_corner, ijk.data(), ijk.size() * sizeof(int), cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(s->rec_w, wt.data(), wt.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemsetAsync(s->traces, 0, (size_t)(nt + 1) * nrec * sizeof(double), s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->nrec = nrec;
  s->nt_rec = nt;
  return FDW_OK;
}

// --------------------------------------------------------------------------
// time loop
// --------------------------------------------------------------------------
extern "C" int fdw_reset(fdw_solver *s) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  DeviceGuard g(s->device);
  const size_t fb = s->d.vol() * s->el;
  const int nf = s->eq == FDW_TTI ? 2 : 1;
  for (int f = 0; f < nf; ++f)
    for (int b = 0; b < 2; ++b) CK(cudaMemsetAsync(s->f[f][b], 0, fb, s->stream));
  if (s->traces) CK(cudaMemsetAsync(s->traces, 0, (size_t)(s->nt_rec + 1) * s->nrec * sizeof(double), s->stream));
  CK(cudaMemsetAsync(s->d_step, 0, sizeof(int), s->stream));
  s->it = 0;
  return FDW_OK;
}

extern "C" int fdw_current_step(const fdw_solver *s) { return s ? s->it : -1; }

extern "C" int fdw_set_current_step(fdw_solver *s, int n) {
  if (!s || n < 0) return fail(FDW_ERR_INVALID_ARG, "bad solver or step");
  DeviceGuard g(s->device);
  CK(cudaMemcpyAsync(s->d_step, &n, sizeof(int), cudaMemcpyHostToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->it = n;
  return FDW_OK;
}

static int ensure_graphs(fdw_solver *s) {
  if (s->graph_ok) return FDW_OK;
  drop_graphs(s);
  int rc = build_maps(s);
  if (rc) return rc;
  // kernel attributes (large dynamic shared memory) are set outside capture
  CK(s->eq == FDW_ACOUSTIC ? acoustic_prepare(s->storage, s->r, s->tile)
                           : tti_prepare(s->storage, s->r, s->tile));
  // per buffer parity b: one step, and a run of kGraphSteps steps (an even
  // number, so the run ends on parity b again); the sparse kernels read the
  // step from the device counter, so a graph serves every step
  for (int b = 0; b < 2; ++b) {
    for (int run = 0; run < 2; ++run) {
      cudaGraph_t gr = nullptr;
      CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
      const int n = run ? kGraphSteps : 1;
      for (int i = 0; i < n && !rc; ++i) rc = enqueue_step(s, (b + i) & 1, s->cap);
      cudaError_t e = cudaStreamEndCapture(s->cap, &gr);
      if (rc) {
        if (gr) cudaGraphDestroy(gr);
        return rc;
      }
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(run ? &s->graph_run[b] : &s->graph[b], gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  s->graph_ok = true;
  return FDW_OK;
}

static int hist_slot_of(const fdw_solver *s, int lvl) {
  const int H = (int)s->hist.size();
  return ((lvl % H) + H) % H;
}

// Steps with the history on (acoustic): level n+1 is written straight into
// its ring slot from the slots of levels n and n-1 (no per-step copy); the
// solver's own two buffers receive the last two levels at the end.
static int step_into_history(fdw_solver *s, int nsteps) {
  CK(acoustic_prepare(s->storage, s->r, s->tile));
  for (int n = 0; n < nsteps; ++n) {
    const int lc = s->it + n, sc = hist_slot_of(s, lc), sp = hist_slot_of(s, lc - 1),
              sn = hist_slot_of(s, lc + 1);
    if (s->hist_level[sc] != lc || s->hist_level[sp] != lc - 1)
      return fail(FDW_ERR_STATE, "history lost levels %d, %d", lc, lc - 1);
    AcousticLaunch L{};
    L.storage = s->storage;
    L.r = s->r;
    L.d = s->d;
    L.w = s->w;
    L.sp = Sponge{s->gam[0], s->gam[1], s->gam[2]};
    L.cur = s->hist[sc];
    L.prev = s->hist[sp];
    L.out = s->hist[sn];
    L.c = s->c;
    L.map_cur_halo = &s->hmap_halo[sc];
    L.map_cur_int = &s->hmap_int[sc];
    L.map_prev_int = &s->hmap_int[sp];
    L.map_c_int = &s->map_c;
    L.zchunks = s->zchunks;
    L.err = s->d_err;
    L.naive = s->naive;
    L.tile = s->tile;
    CK(launch_acoustic(L, s->stream));
    SparseLaunch S{};
    memset(&S, 0, sizeof S);
    S.storage = s->storage;
    S.d = s->d;
    S.sp = L.sp;
    S.f0 = s->hist[sn];
    S.c = s->c;
    S.nsrc = s->nsrc;
    S.src_corner = s->src_corner;
    S.src_w = s->src_w;
    S.wavelet = s->wavelet;
    S.amp_scale = (float)s->fscale;
    S.trace_scale = 1.0 / s->fscale;
    S.nt_src = s->nt_src;
    S.nrec = s->nrec;
    S.rec_corner = s->rec_corner;
    S.rec_w = s->rec_w;
    S.traces = s->traces;
    S.nt_rec = s->nt_rec;
    S.step = s->d_step;
    CK(launch_sparse(S, s->stream));
    s->hist_level[sn] = lc + 1;
  }
  const size_t fb = s->d.vol() * s->el;
  const int last = s->it + nsteps;
  CK(cudaMemcpyAsync(s->f[0][s->cur], s->hist[hist_slot_of(s, last)], fb, cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(s->f[0][1 - s->cur], s->hist[hist_slot_of(s, last - 1)], fb, cudaMemcpyDeviceToDevice,
                     s->stream));
  s->it += nsteps;
  return FDW_OK;
}

extern "C" int fdw_step(fdw_solver *s, int nsteps) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  if (nsteps < 0) return fail(FDW_ERR_INVALID_ARG, "nsteps < 0");
  if (!s->dt_set) return fail(FDW_ERR_STATE, "fdw_set_dt must come before fdw_step");
  if (nsteps == 0) return FDW_OK;
  DeviceGuard g(s->device);
  int rc = ensure_graphs(s);
  if (rc) return rc;
  if (s->hist_on && !s->prof && s->eq == FDW_ACOUSTIC) return step_into_history(s, nsteps);
  const size_t fb = s->d.vol() * s->el;
  for (int n = 0; n < nsteps; ++n) {
    if (!s->prof && !s->hist_on && nsteps - n >= kGraphSteps) {
      // kGraphSteps steps in one launch (the parity is unchanged after it)
      CK(cudaGraphLaunch(s->graph_run[s->cur], s->stream));
      n += kGraphSteps - 1;
      continue;
    }
    if (s->prof && (size_t)(2 * s->prof_n + 1) < s->ev.size()) {
      CK(cudaEventRecord(s->ev[2 * s->prof_n], s->stream));
      rc = enqueue_stencil(s, s->cur, s->stream);
      if (rc) return rc;
      CK(cudaEventRecord(s->ev[2 * s->prof_n + 1], s->stream));
      ++s->prof_n;
      rc = enqueue_sparse(s, s->cur, s->stream);
      if (rc) return rc;
    } else {
      CK(cudaGraphLaunch(s->graph[s->cur], s->stream));
    }
    s->cur = 1 - s->cur;
    if (s->hist_on) {  // keep level it+n+1 for the gradient
      const int lvl = s->it + n + 1, H = (int)s->hist.size();
      const int slot = ((lvl % H) + H) % H;
      CK(cudaMemcpyAsync(s->hist[slot], s->f[0][s->cur], fb, cudaMemcpyDeviceToDevice, s->stream));
      s->hist_level[slot] = lvl;
    }
  }
  s->it += nsteps;
  return FDW_OK;
}

// --------------------------------------------------------------------------
// forward history and adjoint (FWI gradient)
// --------------------------------------------------------------------------
static int check_err_flag(fdw_solver *s);

static int hist_slot(const fdw_solver *s, int lvl) {
  const int H = (int)s->hist.size();
  if (H == 0) return -1;
  const int slot = ((lvl % H) + H) % H;
  return s->hist_level[slot] == lvl ? slot : -1;
}

extern "C" int fdw_history_begin(fdw_solver *s, int nlevels) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  if (s->eq != FDW_ACOUSTIC) return fail(FDW_ERR_INVALID_ARG, "history/adjoint: acoustic only");
  if (nlevels < 3) return fail(FDW_ERR_INVALID_ARG, "nlevels must be >= 3");
  DeviceGuard g(s->device);
  const size_t fb = s->d.vol() * s->el;
  while ((int)s->hist.size() < nlevels) {
    void *p = nullptr;
    CK(cudaMalloc(&p, fb));
    s->hist.push_back(p);
  }
  while ((int)s->hist.size() > nlevels) {
    dfree(s->hist.back());
    s->hist.pop_back();
  }
  s->hist_level.assign(s->hist.size(), INT32_MIN);
  // seed with the two current levels
  const int H = nlevels;
  const int l0 = s->it, l1 = s->it - 1;
  const int s0 = ((l0 % H) + H) % H, s1 = ((l1 % H) + H) % H;
  CK(cudaMemcpyAsync(s->hist[s0], s->f[0][s->cur], fb, cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(s->hist[s1], s->f[0][1 - s->cur], fb, cudaMemcpyDeviceToDevice, s->stream));
  s->hist_level[s0] = l0;
  s->hist_level[s1] = l1;
  // the stencil reads and writes the ring buffers directly (fdw_step)
  TileGeom tg;
  if (acoustic_geom(s->storage, s->r, s->tile, &tg)) return fail(FDW_ERR_INVALID_ARG, "bad tile");
  s->hmap_halo.resize(s->hist.size());
  s->hmap_int.resize(s->hist.size());
  for (size_t i = 0; i < s->hist.size(); ++i) {
    int rc = make_map(&s->hmap_halo[i], s, s->hist[i], tg.box_halo_x, tg.box_halo_y);
    if (!rc) rc = make_map(&s->hmap_int[i], s, s->hist[i], tg.box_int_x, tg.box_int_y);
    if (rc) return rc;
  }
  s->hist_on = true;
  return FDW_OK;
}

extern "C" int fdw_history_end(fdw_solver *s) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  s->hist_on = false;
  return FDW_OK;
}

static int build_adjoint_maps(fdw_solver *s) {
  if (s->amaps_ok) return FDW_OK;
  TileGeom tg;
  if (acoustic_geom(s->storage, s->r, s->tile, &tg)) return fail(FDW_ERR_INVALID_ARG, "bad tile");
  for (int b = 0; b < 2; ++b) {
    int rc = make_map(&s->amap_halo[b], s, s->a[b], tg.box_halo_x, tg.box_halo_y);
    if (rc) return rc;
    rc = make_map(&s->amap_int[b], s, s->a[b], tg.box_int_x, tg.box_int_y);
    if (rc) return rc;
  }
  s->amaps_ok = true;
  return FDW_OK;
}

extern "C" int fdw_adjoint_begin(fdw_solver *s, const double *residual, int nt, int ptr_is_device,
                                 int accumulate_gradient) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  if (s->eq != FDW_ACOUSTIC) return fail(FDW_ERR_INVALID_ARG, "adjoint: acoustic only");
  if (!s->dt_set) return fail(FDW_ERR_STATE, "fdw_set_dt must come before fdw_adjoint_begin");
  if (nt < 0 || (s->nrec > 0 && !residual)) return fail(FDW_ERR_INVALID_ARG, "bad residual");
  DeviceGuard g(s->device);
  const size_t fb = s->d.vol() * s->el;
  for (int b = 0; b < 2; ++b)
    if (!s->a[b]) {
      CK(cudaMalloc(&s->a[b], fb));
      s->amaps_ok = false;
    }
  int rc = build_adjoint_maps(s);
  if (rc) return rc;
  if (!s->d_astep) CK(dmalloc(&s->d_astep, sizeof(int)));
  const size_t rbytes = (size_t)(nt + 1) * (s->nrec > 0 ? s->nrec : 1) * sizeof(double);
  if (s->residual_cap < rbytes) {
    dfree(s->residual);
    s->residual = nullptr;
    CK(dmalloc(&s->residual, rbytes));
    s->residual_cap = rbytes;
  }
  if (s->nrec > 0) {
    rc = upload(s->residual, residual, (size_t)(nt + 1) * s->nrec * sizeof(double), ptr_is_device, s->stream);
    if (rc) return rc;
  }
  s->nt_res = nt;
  dfree(s->src_adj);
  s->src_adj = nullptr;
  if (s->nsrc > 0 && s->nt_src > 0) {
    CK(dmalloc(&s->src_adj, (size_t)s->nt_src * s->nsrc * sizeof(double)));
    CK(cudaMemsetAsync(s->src_adj, 0, (size_t)s->nt_src * s->nsrc * sizeof(double), s->stream));
  }
  for (int b = 0; b < 2; ++b) CK(cudaMemsetAsync(s->a[b], 0, fb, s->stream));
  s->acur = 0;
  s->ak = nt + 1;  // mu_{nt+1} = mu_{nt+2} = 0
  CK(cudaMemcpyAsync(s->d_astep, &s->ak, sizeof(int), cudaMemcpyHostToDevice, s->stream));
  s->adj_grad = accumulate_gradient != 0;
  if (s->adj_grad) {
    if (!s->grad32) CK(dmalloc(&s->grad32, s->d.vol() * sizeof(float)));
    if (!s->grad64) CK(dmalloc(&s->grad64, s->d.vol() * sizeof(double)));
    CK(cudaMemsetAsync(s->grad32, 0, s->d.vol() * sizeof(float), s->stream));
    CK(cudaMemsetAsync(s->grad64, 0, s->d.vol() * sizeof(double), s->stream));
    s->grad_pending = 0;
  }
  CK(cudaStreamSynchronize(s->stream));
  s->adj_on = true;
  return FDW_OK;
}

extern "C" int fdw_adjoint_current_step(const fdw_solver *s) { return s && s->adj_on ? s->ak : -1; }

extern "C" int fdw_adjoint_step(fdw_solver *s, int nsteps) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  if (!s->adj_on) return fail(FDW_ERR_STATE, "fdw_adjoint_begin must come first");
  if (nsteps < 0 || nsteps > s->ak - 1)
    return fail(FDW_ERR_INVALID_ARG, "nsteps must be in [0, %d]", s->ak - 1);
  DeviceGuard g(s->device);
  int rc = acoustic_prepare(s->storage, s->r, s->tile) == cudaSuccess ? FDW_OK : FDW_ERR_CUDA;
  if (rc) return fail(rc, "kernel attribute");
  // A gradient term is held back one step when the next step of this call
  // has one too: the two are added in one pass (both adjoint levels are
  // still in the ping-pong buffers then; the history ring may be refilled
  // after the call, so nothing is held across calls).
  int held = -1;  // level j of the held term j - 1
  for (int n = 0; n < nsteps; ++n) {
    const int cur = s->acur, nxt = 1 - cur;
    const int j = s->ak - 1;  // level produced: mu_j
    AcousticLaunch L{};
    L.storage = s->storage;
    L.r = s->r;
    L.d = s->d;
    L.w = s->w;
    L.sp = Sponge{s->gam[0], s->gam[1], s->gam[2]};
    L.cur = s->a[cur];
    L.prev = s->a[nxt];
    L.c = s->c;
    L.map_cur_halo = &s->amap_halo[cur];
    L.map_cur_int = &s->amap_int[cur];
    L.map_prev_int = &s->amap_int[nxt];
    L.map_c_int = &s->map_c;
    L.zchunks = s->zchunks;
    L.err = s->d_err;
    L.naive = s->naive;
    L.tile = s->tile;
    CK(launch_acoustic(L, s->stream));
    SparseLaunch S{};
    S.storage = s->storage;
    S.d = s->d;
    S.sp = L.sp;
    S.f0 = s->a[nxt];
    S.c = s->c;
    S.nsrc = s->nsrc;
    S.src_corner = s->src_corner;
    S.src_w = s->src_w;
    S.nt_src = s->nt_src;
    S.nrec = s->nrec;
    S.rec_corner = s->rec_corner;
    S.rec_w = s->rec_w;
    S.step = s->d_astep;
    S.residual = s->residual;
    S.nt_res = s->nt_res;
    S.res_scale = (float)(s->h * s->h);
    S.amp_scale = (float)s->fscale;
    S.trace_scale = 1.0 / s->fscale;
    S.adjoint = 1;
    S.src_adj = s->src_adj;
    S.src_adj_scale = (float)(1.0 / (s->h * s->h * s->fscale));
    CK(launch_sparse(S, s->stream));
    if (s->adj_grad && j >= 1) {
      // term n = j - 1: mu_j (P u_j - 2 u_{j-1} + Q u_{j-2}), u_{-1} = 0
      const int s1 = hist_slot(s, j), s0 = hist_slot(s, j - 1), sm = hist_slot(s, j - 2);
      if (s1 < 0 || s0 < 0 || (sm < 0 && j - 2 >= 0))
        return fail(FDW_ERR_STATE, "forward levels %d..%d are not in the history", j - 2, j);
      int added = 0;
      if (held >= 0) {
        // terms held - 1 = j and j - 1: mu_{j+1} (now in a[cur]) and mu_j
        const int sh = hist_slot(s, held);
        if (sh < 0) return fail(FDW_ERR_STATE, "forward level %d is not in the history", held);
        CK(launch_grad_accum_pair(s->storage, s->a[cur], s->a[nxt], s->hist[sh], s->hist[s1], s->hist[s0],
                                  sm >= 0 ? s->hist[sm] : nullptr, s->grad32, s->d, L.sp, s->stream));
        held = -1;
        added = 2;
      } else if (n + 1 < nsteps && j >= 2 && s->grad_pending + 2 <= 64) {
        held = j;  // the next step's term j - 2 joins it
      } else {
        CK(launch_grad_accum(s->storage, s->a[nxt], s->hist[s1], s->hist[s0],
                             sm >= 0 ? s->hist[sm] : nullptr, s->grad32, s->d, L.sp, s->stream));
        added = 1;
      }
      if ((s->grad_pending += added) >= 64) {
        CK(launch_grad_flush(s->grad32, s->grad64, s->d.vol(), s->stream));
        s->grad_pending = 0;
      }
    }
    s->acur = nxt;
    s->ak = j;
  }
  return FDW_OK;
}

extern "C" int fdw_get_gradient(fdw_solver *s, double *grad_m, int ptr_is_device) {
  if (!s || !grad_m) return fail(FDW_ERR_INVALID_ARG, "NULL solver or output");
  if (!s->adj_on || !s->adj_grad) return fail(FDW_ERR_STATE, "no gradient is being accumulated");
  DeviceGuard g(s->device);
  CK(launch_grad_flush(s->grad32, s->grad64, s->d.vol(), s->stream));
  s->grad_pending = 0;
  const size_t n = (size_t)s->nx * s->ny * s->nz;
  double *dst = grad_m;
  if (!ptr_is_device) CK(dmalloc(&dst, n * sizeof(double)));
  cudaError_t e = launch_grad_physical(s->grad64, s->d, s->nx, s->ny, s->nz, s->nb,
                                       -1.0 / (s->dt * s->dt * s->fscale * s->fscale), dst,
                                       s->stream);
  if (e == cudaSuccess && !ptr_is_device) {
    e = cudaMemcpyAsync(grad_m, dst, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(dst);
  }
  if (e != cudaSuccess) return cuda_fail(e, "fdw_get_gradient");
  return ptr_is_device ? FDW_OK : check_err_flag(s);
}

extern "C" int fdw_get_source_adjoint(fdw_solver *s, double *out, int ptr_is_device) {
  if (!s || !out) return fail(FDW_ERR_INVALID_ARG, "NULL solver or output");
  if (!s->adj_on || !s->src_adj) return fail(FDW_ERR_STATE, "no source adjoint (no sources or no adjoint run)");
  DeviceGuard g(s->device);
  const size_t bytes = (size_t)s->nt_src * s->nsrc * sizeof(double);
  CK(cudaMemcpyAsync(out, s->src_adj, bytes, ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     s->stream));
  if (!ptr_is_device) return check_err_flag(s);
  return FDW_OK;
}

extern "C" int fdw_get_adjoint_wavefield(const fdw_solver *cs, int level, float *out, int ptr_is_device) {
  fdw_solver *s = (fdw_solver *)cs;
  if (!s || !out || level < 0 || level > 1) return fail(FDW_ERR_INVALID_ARG, "bad arguments");
  if (!s->adj_on) return fail(FDW_ERR_STATE, "no adjoint run");
  DeviceGuard g(s->device);
  const size_t n = (size_t)s->d.NX * s->d.NY * s->d.NZ;
  float *dst = out;
  if (!ptr_is_device) CK(dmalloc(&dst, n * sizeof(float)));
  cudaError_t e = launch_unpack(s->storage, s->a[level == 0 ? s->acur : 1 - s->acur], s->d, dst,
                                (float)(1.0 / s->fscale), s->stream);
  if (e == cudaSuccess && !ptr_is_device) {
    e = cudaMemcpyAsync(out, dst, n * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(dst);
  }
  if (e != cudaSuccess) return cuda_fail(e, "fdw_get_adjoint_wavefield");
  return FDW_OK;
}

extern "C" int fdw_step_closure(fdw_solver *s, fdw_closure *c, int nsteps) {
  return fdw_step_closure_every(s, c, nsteps, 1);
}

extern "C" int fdw_step_closure_every(fdw_solver *s, fdw_closure *c, int nsteps, int every) {
  if (!s || !c) return fail(FDW_ERR_INVALID_ARG, "NULL solver or closure");
  if (s->eq != FDW_ACOUSTIC) return fail(FDW_ERR_INVALID_ARG, "the closure corrects the acoustic step");
  if (nsteps < 0) return fail(FDW_ERR_INVALID_ARG, "nsteps < 0");
  if (every < 1) return fail(FDW_ERR_INVALID_ARG, "every must be >= 1");
  if (!s->dt_set) return fail(FDW_ERR_STATE, "fdw_set_dt must come before fdw_step_closure");
  DeviceGuard g(s->device);
  int rc = build_maps(s);
  if (rc) return rc;
  CK(acoustic_prepare(s->storage, s->r, s->tile));
  if (closure_reserve_infer(c, s->d)) return fail(FDW_ERR_OOM, "closure inference workspace");
  if (nsteps > 0)  // the network's answer for a zero wavefield, subtracted every step
    CK(closure_infer_base(c, s->vp, s->nx, s->ny, s->nz, s->nb, s->d, s->d_err, s->stream));
  const size_t fb = s->d.vol() * s->el;
  for (int n = 0; n < nsteps; ++n) {
    const int cur = s->cur, nxt = 1 - cur;
    // the phase follows the solver's step count, so chunked calls correct
    // the same steps as one call over the same interval
    const bool corr = ((s->it + n) % every) == 0;
    if (corr)
      CK(closure_infer_pre(c, s->storage, s->f[0][cur], s->f[0][nxt], s->vp, s->nx, s->ny, s->nz, s->nb,
                           s->d, s->d_err, s->stream));
    rc = enqueue_stencil(s, cur, s->stream);
    if (rc) return rc;
    if (corr)
      CK(closure_infer_apply(c, s->storage, s->f[0][nxt], s->d, s->nx, s->ny, s->nz, s->nb, (float)every,
                             s->stream));
    rc = enqueue_sparse(s, cur, s->stream);
    if (rc) return rc;
    s->cur = nxt;
    if (s->hist_on) {
      const int lvl = s->it + n + 1, H = (int)s->hist.size();
      const int slot = ((lvl % H) + H) % H;
      CK(cudaMemcpyAsync(s->hist[slot], s->f[0][s->cur], fb, cudaMemcpyDeviceToDevice, s->stream));
      s->hist_level[slot] = lvl;
    }
  }
  s->it += nsteps;
  return FDW_OK;
}

extern "C" int fdw_profile_begin(fdw_solver *s, int max_launches) {
  if (!s || max_launches < 1 || max_launches > 65536)
    return fail(FDW_ERR_INVALID_ARG, "max_launches must be in [1, 65536]");
  DeviceGuard g(s->device);
  const size_t need = 2 * (size_t)max_launches;
  while (s->ev.size() < need) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    s->ev.push_back(e);
  }
  s->prof = true;
  s->prof_n = 0;
  return FDW_OK;
}

extern "C" int fdw_profile_end(fdw_solver *s, double *stencil_ms, int *launches) {
  if (!s || !stencil_ms || !launches) return fail(FDW_ERR_INVALID_ARG, "NULL argument");
  if (!s->prof) return fail(FDW_ERR_STATE, "fdw_profile_begin was not called");
  DeviceGuard g(s->device);
  CK(cudaStreamSynchronize(s->stream));
  double tot = 0.0;
  for (int i = 0; i < s->prof_n; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, s->ev[2 * i], s->ev[2 * i + 1]));
    tot += ms;
  }
  *stencil_ms = tot;
  *launches = s->prof_n;
  s->prof = false;
  s->prof_n = 0;
  return FDW_OK;
}

// --------------------------------------------------------------------------
// outputs, state, checks
// --------------------------------------------------------------------------
static int check_err_flag(fdw_solver *s) {
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (flag) {
    CK(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
    if (flag & kErrWaitTimeout)
      return fail(FDW_ERR_DEVICE_TIMEOUT, "a kernel gave up waiting for its TMA copies (flag %d)", flag);
    return fail(FDW_ERR_CUDA, "device error flag %d", flag);
  }
  return FDW_OK;
}

extern "C" int fdw_gather_receivers(fdw_solver *s, double *out, int ptr_is_device) {
  if (!s || !out) return fail(FDW_ERR_INVALID_ARG, "NULL solver or output");
  if (!s->traces) return fail(FDW_ERR_STATE, "no receivers set");
  DeviceGuard g(s->device);
  const size_t bytes = (size_t)(s->nt_rec + 1) * s->nrec * sizeof(double);
  CK(cudaMemcpyAsync(out, s->traces, bytes, ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     s->stream));
  if (!ptr_is_device) return check_err_flag(s);
  return FDW_OK;
}

static void *level_ptr(const fdw_solver *s, int field, int level) {
  const int b = level == 0 ? s->cur : 1 - s->cur;
  return s->f[field][b];
}

extern "C" int fdw_get_wavefield(const fdw_solver *cs, int field, int level, float *out, int ptr_is_device) {
  fdw_solver *s = (fdw_solver *)cs;
  if (!s || !out) return fail(FDW_ERR_INVALID_ARG, "NULL solver or output");
  if (field < 0 || field > (s->eq == FDW_TTI ? 1 : 0) || level < 0 || level > 1)
    return fail(FDW_ERR_INVALID_ARG, "bad field/level");
  DeviceGuard g(s->device);
  const size_t n = (size_t)s->d.NX * s->d.NY * s->d.NZ;
  float *dst = out;
  if (!ptr_is_device) CK(dmalloc(&dst, n * sizeof(float)));
  cudaError_t e = launch_unpack(s->storage, level_ptr(s, field, level), s->d, dst,
                                (float)(1.0 / s->fscale), s->stream);
  if (e == cudaSuccess && !ptr_is_device) {
    e = cudaMemcpyAsync(out, dst, n * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(dst);
  }
  if (e != cudaSuccess) return cuda_fail(e, "fdw_get_wavefield");
  return FDW_OK;
}

extern "C" int fdw_set_wavefield(fdw_solver *s, int field, int level, const float *in, int ptr_is_device) {
  if (!s || !in) return fail(FDW_ERR_INVALID_ARG, "NULL solver or input");
  if (field < 0 || field > (s->eq == FDW_TTI ? 1 : 0) || level < 0 || level > 1)
    return fail(FDW_ERR_INVALID_ARG, "bad field/level");
  DeviceGuard g(s->device);
  const size_t n = (size_t)s->d.NX * s->d.NY * s->d.NZ;
  const float *src = in;
  float *tmp = nullptr;
  if (!ptr_is_device) {
    CK(dmalloc(&tmp, n * sizeof(float)));
    cudaError_t e = cudaMemcpyAsync(tmp, in, n * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) {
      cudaFree(tmp);
      return cuda_fail(e, "fdw_set_wavefield copy");
    }
    src = tmp;
  }
  cudaError_t e = launch_pack(s->storage, src, level_ptr(s, field, level), s->d, (float)s->fscale,
                              s->stream);
  if (tmp) {
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(tmp);
  }
  if (e != cudaSuccess) return cuda_fail(e, "fdw_set_wavefield");
  return FDW_OK;
}

extern "C" int fdw_check(fdw_solver *s, int check_finite) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  DeviceGuard g(s->device);
  int rc = check_err_flag(s);
  if (rc) return rc;
  if (check_finite) {
    CK(cudaMemsetAsync(s->scratch2, 0, sizeof(int), s->stream));
    const int nf = s->eq == FDW_TTI ? 2 : 1;
    for (int f = 0; f < nf; ++f)
      for (int b = 0; b < 2; ++b) CK(launch_nonfinite(s->storage, s->f[f][b], s->d, (int *)s->scratch2, s->stream));
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, s->scratch2, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (flag) return fail(FDW_ERR_DIVERGED, "non-finite values in the wavefield at step %d", s->it);
  }
  return FDW_OK;
}

extern "C" int fdw_set_field_scale(fdw_solver *s, double scale) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  if (!(scale >= 0.0) || !isfinite(scale)) return fail(FDW_ERR_INVALID_ARG, "scale must be >= 0");
  s->fscale_req = scale;
  s->dt_set = false;
  drop_graphs(s);
  return FDW_OK;
}

extern "C" double fdw_get_field_scale(const fdw_solver *s) { return s ? s->fscale : -1.0; }

extern "C" int fdw_set_sponge(fdw_solver *s, double vref, double R) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  if (!isfinite(vref) || !(R > 0.0 && R < 1.0)) return fail(FDW_ERR_INVALID_ARG, "need finite vref, 0 < R < 1");
  s->sponge_vref = vref;
  s->sponge_R = R;
  s->dt_set = false;
  drop_graphs(s);
  return FDW_OK;
}

extern "C" int fdw_set_kernel_variant(fdw_solver *s, int variant) {
  if (!s || variant < 0 || variant > 1) return fail(FDW_ERR_INVALID_ARG, "variant must be 0 or 1");
  s->naive = variant;
  drop_graphs(s);
  return FDW_OK;
}

extern "C" int fdw_set_tile_config(fdw_solver *s, int tile) {
  if (!s) return fail(FDW_ERR_INVALID_ARG, "NULL solver");
  TileGeom tg;
  const bool tti = s->eq == FDW_TTI;
  const int ntiles = tti ? kTtiTilesMax : kAcTiles;
  if (tile < -1 || tile >= ntiles ||
      (tile >= 0 && (tti ? tti_geom(s->storage, s->r, tile, &tg) : acoustic_geom(s->storage, s->r, tile, &tg))))
    return fail(FDW_ERR_INVALID_ARG, "tile configuration must be -1 (default) or 0..%d", ntiles - 1);
  s->tile = tile >= 0 ? tile : tti ? tti_default_tile(s->storage, s->r) : acoustic_default_tile(s->storage, s->r);
  s->maps_ok = false;
  s->zchunks = default_zchunks(s);
  drop_graphs(s);
  return FDW_OK;
}

extern "C" int fdw_get_tile_config(const fdw_solver *s) { return s ? s->tile : -1; }

extern "C" int fdw_set_zchunks(fdw_solver *s, int zchunks) {
  if (!s || zchunks < 0) return fail(FDW_ERR_INVALID_ARG, "zchunks must be >= 0");
  if (zchunks > 0 && zchunks < min_zchunks(s))
    return fail(FDW_ERR_INVALID_ARG, "zchunks must be >= %d (at most %d planes per CTA)",
                min_zchunks(s), kMaxZChunk);
  s->zchunks = zchunks == 0 ? default_zchunks(s) : zchunks;
  drop_graphs(s);
  return FDW_OK;
}

extern "C" int fdw_get_zchunks(const fdw_solver *s) { return s ? s->zchunks : -1; }
