// setup.cu -- one-off kernels: medium coefficients on the computational
// grid, velocity maxima, field (un)packing, the non-finite watchdog.
#include "fdw_internal.h"
#include "fdwave.h"

namespace fdw {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Medium extension into the sponge: a computational point takes the value
// of the nearest physical point.

// c' = (v dt/h)^2 in FP32 arithmetic accurate to a few ulp: dt/h as an
// unevaluated sum hi + lo of two floats, v (hi + lo) = p + e exactly enough
// (fmaf gives the rounding error of v hi), then (p + e)^2 ~ p^2 + 2 p e with
// one rounding. (Computing it in FP64 made this set-up kernel take 1.6 ms at
// 592^3: FP64 runs at a small fraction of the FP32 rate on this part.)
__device__ __forceinline__ float coef_of(float v, float hi, float lo) {
  const float p = v * hi;
  const float e = fmaf(v, hi, -p) + v * lo;
  return fmaf(p, p, 2.f * p * e);
}

// The field kernels walk rows: a block takes rows (j, k) of the padded
// layout in turn and its threads the x points of a row, so the index
// arithmetic is one division per row.
template <typename T>
__global__ void coef_acoustic_kernel(const float *__restrict__ vp, int nx, int ny, int nz, int nb,
                                     Dims d, double dt_over_h, T *__restrict__ c) {
  const float hi = (float)dt_over_h, lo = (float)(dt_over_h - (double)hi);
  const int rows = d.NY * d.NZ;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % d.NY, k = row / d.NY;
    T *cr = c + (size_t)row * d.Xp;
    const float *vr = vp + ((size_t)clampi(k - nb, 0, nz - 1) * ny + clampi(j - nb, 0, ny - 1)) * nx;
    for (int i = threadIdx.x; i < d.Xp; i += blockDim.x)
      cr[i] = St<T>::st(i < d.NX ? coef_of(vr[clampi(i - nb, 0, nx - 1)], hi, lo) : 0.f);
  }
}

// The next smaller value of a positive finite number of the storage type.
__device__ __forceinline__ float ulp_down(float v) { return __uint_as_float(__float_as_uint(v) - 1u); }
__device__ __forceinline__ __nv_bfloat16 ulp_down(__nv_bfloat16 v) {
  return __ushort_as_bfloat16((unsigned short)(__bfloat16_as_ushort(v) - 1u));
}
__device__ __forceinline__ __half ulp_down(__half v) {
  return __ushort_as_half((unsigned short)(__half_as_ushort(v) - 1u));
}

template <typename T>
__global__ void coef_tti_kernel(const float *__restrict__ vp, const float *__restrict__ eps,
                                const float *__restrict__ delta, const float *__restrict__ theta,
                                const float *__restrict__ phi, int nx, int ny, int nz, int nb,
                                Dims d, double dt_over_h, T *c, T *e, T *dl, T *ax, T *ay) {
  const float hi = (float)dt_over_h, lo = (float)(dt_over_h - (double)hi);
  const int rows = d.NY * d.NZ;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % d.NY, k = row / d.NY;
    const size_t pr = ((size_t)clampi(k - nb, 0, nz - 1) * ny + clampi(j - nb, 0, ny - 1)) * nx;
    for (int i = threadIdx.x; i < d.Xp; i += blockDim.x) {
      const size_t p = (size_t)row * d.Xp + i;
      float vc = 0.f, ve = 0.f, vd = 0.f, vx = 0.f, vy = 0.f;
      if (i < d.NX) {
        // FP32 arithmetic (FP64 is slow here): each value within a few ulp
        const size_t q = pr + clampi(i - nb, 0, nx - 1);
        vc = coef_of(vp[q], hi, lo);
        ve = fmaf(2.f, eps[q], 1.f);
        vd = sqrtf(fmaf(2.f, delta[q], 1.f));
        float st, ct, sp, cp;
        sincosf(theta[q], &st, &ct);
        sincosf(phi[q], &sp, &cp);
        float sx = st * cp, sy = st * sp;
        if (ct < 0.f) { sx = -sx; sy = -sy; }  // n and -n give the same operator
        vx = sx;
        vy = sy;
      }
      c[p] = St<T>::st(vc);
      // The rounded pair must keep the system matrix [[e, d], [d, 1]] of
      // Eq. TTI positive semidefinite (e >= d^2, i.e. eps >= delta, which
      // the model may meet with equality): rounding e and d independently
      // can give d^2 > e by an ulp of the storage type -- a local
      // instability that 16-bit storage turns into growth. d is moved down
      // by ulps until e >= d^2 holds exactly for the stored values.
      const T es = St<T>::st(ve);
      T ds = St<T>::st(vd);
      for (int it = 0; it < 8 && (double)St<T>::ld(ds) * (double)St<T>::ld(ds) > (double)St<T>::ld(es); ++it)
        ds = ulp_down(ds);
      e[p] = es;
      dl[p] = ds;
      ax[p] = St<T>::st(vx);
      ay[p] = St<T>::st(vy);
    }
  }
}

// out[0] = max v, out[1] = max v sqrt(1 + 2 eps), out[2] = flag of a
// non-positive or non-finite v, out[3] = max (1 - |cos theta|) (steepest
// tilt); out must be zeroed (all maxima are of non-negative values).
__global__ void max_velocity_kernel(const float *__restrict__ vp, const float *__restrict__ eps,
                                    const float *__restrict__ theta, long n, float *out) {
  float m0 = 0.f, m1 = 0.f, m3 = 0.f;
  int bad = 0;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x) {
    const float v = vp[p];
    bad |= !(v > 0.f) || !isfinite(v);
    m0 = fmaxf(m0, v);
    m1 = fmaxf(m1, eps ? v * sqrtf(1.f + 2.f * eps[p]) : v);
    if (theta) m3 = fmaxf(m3, 1.f - fabsf(cosf(theta[p])));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    m3 = fmaxf(m3, __shfl_xor_sync(0xffffffffu, m3, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax((int *)&out[0], __float_as_int(m0));
    atomicMax((int *)&out[1], __float_as_int(m1));
    if (bad) atomicOr((int *)&out[2], 1);
    atomicMax((int *)&out[3], __float_as_int(m3));
  }
}

template <typename T>
__global__ void pack_kernel(const float *__restrict__ src, T *__restrict__ dst, Dims d, float scale) {
  const int rows = d.NY * d.NZ;
  for (int row = blockIdx.x; row < rows; row += gridDim.x)
    for (int i = threadIdx.x; i < d.Xp; i += blockDim.x)
      dst[(size_t)row * d.Xp + i] = St<T>::st(i < d.NX ? scale * src[(size_t)row * d.NX + i] : 0.f);
}

template <typename T>
__global__ void unpack_kernel(const T *__restrict__ src, float *__restrict__ dst, Dims d, float scale) {
  const int rows = d.NY * d.NZ;
  for (int row = blockIdx.x; row < rows; row += gridDim.x)
    for (int i = threadIdx.x; i < d.NX; i += blockDim.x)
      dst[(size_t)row * d.NX + i] = scale * St<T>::ld(src[(size_t)row * d.Xp + i]);
}

// (padding columns hold zeros, so the whole padded volume is scanned flat)
template <typename T>
__global__ void nonfinite_kernel(const T *__restrict__ f, size_t n, int *flag) {
  int bad = 0;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(St<T>::ld(f[p]));
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// one block per row (rows of a computational grid; capped)
static int row_grid(const Dims &d) {
  const long r = (long)d.NY * d.NZ;
  return (int)(r < 152 * 64 ? (r < 1 ? 1 : r) : 152 * 64);
}

static int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

#define FDW_DISPATCH(storage, KERNEL_CALL)                    \
  switch (storage) {                                          \
    case FDW_F32: { using T = float; KERNEL_CALL; break; }    \
    case FDW_BF16: { using T = __nv_bfloat16; KERNEL_CALL; break; } \
    case FDW_F16: { using T = __half; KERNEL_CALL; break; }   \
    default: return cudaErrorInvalidValue;                    \
  }

cudaError_t launch_coef_acoustic(int storage, const float *vp, int nx, int ny, int nz, int nb,
                                 Dims d, double dt_over_h, void *c, cudaStream_t st) {
  FDW_DISPATCH(storage, (coef_acoustic_kernel<T><<<row_grid(d), 256, 0, st>>>(
                            vp, nx, ny, nz, nb, d, dt_over_h, (T *)c)));
  return cudaGetLastError();
}

cudaError_t launch_coef_tti(int storage, const float *vp, const float *eps, const float *delta,
                            const float *theta, const float *phi, int nx, int ny, int nz, int nb,
                            Dims d, double dt_over_h, void *c, void *e, void *dl, void *ax,
                            void *ay, cudaStream_t st) {
  FDW_DISPATCH(storage, (coef_tti_kernel<T><<<row_grid(d), 256, 0, st>>>(
                            vp, eps, delta, theta, phi, nx, ny, nz, nb, d, dt_over_h, (T *)c,
                            (T *)e, (T *)dl, (T *)ax, (T *)ay)));
  return cudaGetLastError();
}

cudaError_t launch_max_velocity(const float *vp, const float *eps, const float *theta, long n, float *out4,
                                cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out4, 0, 4 * sizeof(float), st);
  if (e != cudaSuccess) return e;
  max_velocity_kernel<<<grid_for((size_t)n), 256, 0, st>>>(vp, eps, theta, n, out4);
  return cudaGetLastError();
}

cudaError_t launch_pack(int storage, const float *src, void *dst, Dims d, float scale,
                        cudaStream_t st) {
  FDW_DISPATCH(storage, (pack_kernel<T><<<row_grid(d), 256, 0, st>>>(src, (T *)dst, d, scale)));
  return cudaGetLastError();
}

cudaError_t launch_unpack(int storage, const void *src, Dims d, float *dst, float scale,
                          cudaStream_t st) {
  FDW_DISPATCH(storage, (unpack_kernel<T><<<row_grid(d), 256, 0, st>>>(
                            (const T *)src, dst, d, scale)));
  return cudaGetLastError();
}

cudaError_t launch_nonfinite(int storage, const void *f, Dims d, int *flag, cudaStream_t st) {
  FDW_DISPATCH(storage, (nonfinite_kernel<T><<<grid_for(d.vol()), 256, 0, st>>>(
                            (const T *)f, d.vol(), flag)));
  return cudaGetLastError();
}

}  // namespace fdw
