// setup.cu -- one-off kernels: medium coefficients on the computational
// grid, velocity maxima, field (un)packing, the non-finite watchdog.
#include "fdw_internal.h"
#include "fdwave.h"

namespace fdw {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Medium extension into the sponge: a computational point takes the value
// of the nearest physical point.
__device__ __forceinline__ size_t phys_index(int i, int j, int k, int nx, int ny, int nz, int nb) {
  const int pi = clampi(i - nb, 0, nx - 1), pj = clampi(j - nb, 0, ny - 1), pk = clampi(k - nb, 0, nz - 1);
  return ((size_t)pk * ny + pj) * nx + pi;
}

template <typename T>
__global__ void coef_acoustic_kernel(const float *__restrict__ vp, int nx, int ny, int nz, int nb,
                                     Dims d, double dt_over_h, T *__restrict__ c) {
  const size_t n = d.vol();
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n;
       p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % d.Xp);
    const size_t rest = p / d.Xp;
    const int j = (int)(rest % d.NY), k = (int)(rest / d.NY);
    float v = 0.f;
    if (i < d.NX) {
      const double cv = (double)vp[phys_index(i, j, k, nx, ny, nz, nb)] * dt_over_h;
      v = (float)(cv * cv);
    }
    c[p] = St<T>::st(v);
  }
}

template <typename T>
__global__ void coef_tti_kernel(const float *__restrict__ vp, const float *__restrict__ eps,
                                const float *__restrict__ delta, const float *__restrict__ theta,
                                const float *__restrict__ phi, int nx, int ny, int nz, int nb,
                                Dims d, double dt_over_h, T *c, T *e, T *dl, T *ax, T *ay) {
  const size_t n = d.vol();
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n;
       p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % d.Xp);
    const size_t rest = p / d.Xp;
    const int j = (int)(rest % d.NY), k = (int)(rest / d.NY);
    float vc = 0.f, ve = 0.f, vd = 0.f, vx = 0.f, vy = 0.f;
    if (i < d.NX) {
      const size_t q = phys_index(i, j, k, nx, ny, nz, nb);
      const double cv = (double)vp[q] * dt_over_h;
      vc = (float)(cv * cv);
      ve = (float)(1.0 + 2.0 * (double)eps[q]);
      vd = (float)sqrt(1.0 + 2.0 * (double)delta[q]);
      const double th = theta[q], ph = phi[q];
      double sx = sin(th) * cos(ph), sy = sin(th) * sin(ph);
      if (cos(th) < 0.0) { sx = -sx; sy = -sy; }  // n and -n give the same operator
      vx = (float)sx;
      vy = (float)sy;
    }
    c[p] = St<T>::st(vc);
    e[p] = St<T>::st(ve);
    dl[p] = St<T>::st(vd);
    ax[p] = St<T>::st(vx);
    ay[p] = St<T>::st(vy);
  }
}

// out[0] = max vp, out[1] = max vp sqrt(1 + 2 eps) (eps may be null), as
// float bits (positive floats order like their bit patterns); out[2] = 1 if
// some vp is not a positive finite number.
__global__ void max_velocity_kernel(const float *__restrict__ vp, const float *__restrict__ eps,
                                    long n, float *out) {
  float m0 = 0.f, m1 = 0.f;
  int bad = 0;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x) {
    const float v = vp[p];
    bad |= !(v > 0.f) || !isfinite(v);
    m0 = fmaxf(m0, v);
    m1 = fmaxf(m1, eps ? v * sqrtf(1.f + 2.f * eps[p]) : v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax((int *)&out[0], __float_as_int(m0));
    atomicMax((int *)&out[1], __float_as_int(m1));
    if (bad) atomicOr((int *)&out[2], 1);
  }
}

template <typename T>
__global__ void pack_kernel(const float *__restrict__ src, T *__restrict__ dst, Dims d, float scale) {
  const size_t n = d.vol();
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n;
       p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % d.Xp);
    const size_t row = p / d.Xp;
    dst[p] = St<T>::st(i < d.NX ? scale * src[row * d.NX + i] : 0.f);
  }
}

template <typename T>
__global__ void unpack_kernel(const T *__restrict__ src, float *__restrict__ dst, Dims d, float scale) {
  const size_t n = (size_t)d.NX * d.NY * d.NZ;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n;
       p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % d.NX);
    const size_t row = p / d.NX;
    dst[p] = scale * St<T>::ld(src[row * d.Xp + i]);
  }
}

template <typename T>
__global__ void nonfinite_kernel(const T *__restrict__ f, Dims d, int *flag) {
  const size_t n = d.vol();
  int bad = 0;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n;
       p += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(St<T>::ld(f[p]));
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
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
  FDW_DISPATCH(storage, (coef_acoustic_kernel<T><<<grid_for(d.vol()), 256, 0, st>>>(
                            vp, nx, ny, nz, nb, d, dt_over_h, (T *)c)));
  return cudaGetLastError();
}

cudaError_t launch_coef_tti(int storage, const float *vp, const float *eps, const float *delta,
                            const float *theta, const float *phi, int nx, int ny, int nz, int nb,
                            Dims d, double dt_over_h, void *c, void *e, void *dl, void *ax,
                            void *ay, cudaStream_t st) {
  FDW_DISPATCH(storage, (coef_tti_kernel<T><<<grid_for(d.vol()), 256, 0, st>>>(
                            vp, eps, delta, theta, phi, nx, ny, nz, nb, d, dt_over_h, (T *)c,
                            (T *)e, (T *)dl, (T *)ax, (T *)ay)));
  return cudaGetLastError();
}

cudaError_t launch_max_velocity(const float *vp, const float *eps, long n, float *out3,
                                cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out3, 0, 3 * sizeof(float), st);
  if (e != cudaSuccess) return e;
  max_velocity_kernel<<<grid_for((size_t)n), 256, 0, st>>>(vp, eps, n, out3);
  return cudaGetLastError();
}

cudaError_t launch_pack(int storage, const float *src, void *dst, Dims d, float scale,
                        cudaStream_t st) {
  FDW_DISPATCH(storage, (pack_kernel<T><<<grid_for(d.vol()), 256, 0, st>>>(src, (T *)dst, d, scale)));
  return cudaGetLastError();
}

cudaError_t launch_unpack(int storage, const void *src, Dims d, float *dst, float scale,
                          cudaStream_t st) {
  FDW_DISPATCH(storage, (unpack_kernel<T><<<grid_for((size_t)d.NX * d.NY * d.NZ), 256, 0, st>>>(
                            (const T *)src, dst, d, scale)));
  return cudaGetLastError();
}

cudaError_t launch_nonfinite(int storage, const void *f, Dims d, int *flag, cudaStream_t st) {
  FDW_DISPATCH(storage, (nonfinite_kernel<T><<<grid_for(d.vol()), 256, 0, st>>>(
                            (const T *)f, d, flag)));
  return cudaGetLastError();
}

}  // namespace fdw
