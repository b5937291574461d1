// adjoint.cu -- FWI gradient kernels.
//
// The paper motivates the solvers by FWI/RTM (Introduction); the gradient
// is the transpose of the discrete recurrence of Algorithm 1 / Eq. Acou
// with the sponge. With the forward recurrence
//   P u_{n+1} = (2 + C L) u_n - Q u_{n-1} + C q_n,   C = dt^2 v^2 = dt^2 / m,
// and multipliers mu produced by the same step run backwards (fdw_adjoint_*),
//   dJ/dm = -(1/dt^2) sum_n mu_{n+1} (P u_{n+1} - 2 u_n + Q u_{n-1}).
// grad_accum adds one term in FP32 (a segment of steps), grad_flush moves
// the FP32 partial sums into the FP64 total, grad_physical applies the
// -1/dt^2 scale and the adjoint of the medium's extension into the sponge
// (each physical point collects every computational point that copies it).
#include "fdw_internal.h"
#include "fdwave.h"

namespace fdw {

// One block per row (j, k) of the padded layout, threads along x: the
// damping of the row is loaded once and no 64-bit division is done per
// point (that index arithmetic made this per-step kernel issue-bound). Used
// for grids of 2^31 or more groups of four points; grad_accum4_kernel below
// otherwise.
template <typename T>
__global__ void grad_accum_kernel(const T *__restrict__ mu, const T *__restrict__ u1,
                                  const T *__restrict__ u0, const T *__restrict__ um1,
                                  float *__restrict__ g32, Dims d, Sponge sp) {
  const int rows = d.NY * d.NZ;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % d.NY, k = row / d.NY;
    const float gyz = sp.gy[j] + sp.gz[k];
    const size_t base = (size_t)row * d.Xp;
    for (int i = threadIdx.x; i < d.NX; i += blockDim.x) {
      const size_t p = base + i;
      const float gh = sp.gx[i] + gyz;
      const float a = St<T>::ld(mu[p]);
      const float b = (1.f + gh) * St<T>::ld(u1[p]) - 2.f * St<T>::ld(u0[p]) +
                      (um1 ? (1.f - gh) * St<T>::ld(um1[p]) : 0.f);
      g32[p] = fmaf(a, b, g32[p]);
    }
  }
}

// The same term four points at a time (the padded row length is a multiple
// of 32): 16-byte loads of the fields and of the FP32 partial sum, one 32-bit
// division per four points for the row index. Points of the row padding
// (x >= NX) are skipped.
template <typename T>
__global__ void __launch_bounds__(256)
    grad_accum4_kernel(const T *__restrict__ mu, const T *__restrict__ u1, const T *__restrict__ u0,
                       const T *__restrict__ um1, float *__restrict__ g32, Dims d, Sponge sp, int nq) {
  using V = struct alignas(4 * sizeof(T)) { T v[4]; };
  const int xq = d.Xp / 4;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const int row = q / xq, i0 = (q - row * xq) * 4;
    if (i0 >= d.NX) continue;
    const int j = row % d.NY, k = row / d.NY;
    const float gyz = sp.gy[j] + sp.gz[k];
    const V a = reinterpret_cast<const V *>(mu)[q];
    const V b1 = reinterpret_cast<const V *>(u1)[q];
    const V b0 = reinterpret_cast<const V *>(u0)[q];
    V bm;
    if (um1) bm = reinterpret_cast<const V *>(um1)[q];
    float4 g = reinterpret_cast<float4 *>(g32)[q];
    float *ge = reinterpret_cast<float *>(&g);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (i0 + e < d.NX) {
        const float gh = sp.gx[i0 + e] + gyz;
        const float b = (1.f + gh) * St<T>::ld(b1.v[e]) - 2.f * St<T>::ld(b0.v[e]) +
                        (um1 ? (1.f - gh) * St<T>::ld(bm.v[e]) : 0.f);
        ge[e] = fmaf(St<T>::ld(a.v[e]), b, ge[e]);
      }
    }
    reinterpret_cast<float4 *>(g32)[q] = g;
  }
}

// Two consecutive terms in one pass, four points at a time: term j-1,
// mu_j (P u_j - 2 u_{j-1} + Q u_{j-2}), then term j-2, mu_{j-1} (P u_{j-1}
// - 2 u_{j-2} + Q u_{j-3}) (u_{j-3} = 0 when absent), added in that order
// as the single-term kernel would over two steps; the partial sum and the
// shared levels are read once instead of twice.
template <typename T>
__global__ void __launch_bounds__(256)
    grad_accum4_pair_kernel(const T *__restrict__ mu_a, const T *__restrict__ mu_b, const T *__restrict__ ua,
                            const T *__restrict__ ub, const T *__restrict__ uc, const T *__restrict__ ud,
                            float *__restrict__ g32, Dims d, Sponge sp, int nq) {
  using V = struct alignas(4 * sizeof(T)) { T v[4]; };
  const int xq = d.Xp / 4;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const int row = q / xq, i0 = (q - row * xq) * 4;
    if (i0 >= d.NX) continue;
    const int j = row % d.NY, k = row / d.NY;
    const float gyz = sp.gy[j] + sp.gz[k];
    const V ma = reinterpret_cast<const V *>(mu_a)[q];
    const V mb = reinterpret_cast<const V *>(mu_b)[q];
    const V a = reinterpret_cast<const V *>(ua)[q];
    const V b = reinterpret_cast<const V *>(ub)[q];
    const V c = reinterpret_cast<const V *>(uc)[q];
    V dd;
    if (ud) dd = reinterpret_cast<const V *>(ud)[q];
    float4 g = reinterpret_cast<float4 *>(g32)[q];
    float *ge = reinterpret_cast<float *>(&g);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (i0 + e < d.NX) {
        const float gh = sp.gx[i0 + e] + gyz;
        const float t1 = (1.f + gh) * St<T>::ld(a.v[e]) - 2.f * St<T>::ld(b.v[e]) + (1.f - gh) * St<T>::ld(c.v[e]);
        const float t2 = (1.f + gh) * St<T>::ld(b.v[e]) - 2.f * St<T>::ld(c.v[e]) +
                         (ud ? (1.f - gh) * St<T>::ld(dd.v[e]) : 0.f);
        ge[e] = fmaf(St<T>::ld(mb.v[e]), t2, fmaf(St<T>::ld(ma.v[e]), t1, ge[e]));
      }
    }
    reinterpret_cast<float4 *>(g32)[q] = g;
  }
}

__global__ void grad_flush_kernel(float *__restrict__ g32, double *__restrict__ g64, size_t n) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n;
       p += (size_t)gridDim.x * blockDim.x) {
    g64[p] += (double)g32[p];
    g32[p] = 0.f;
  }
}

// out[pk][pj][pi] (physical grid) = scale * sum of g64 over the
// computational points whose medium is copied from (pi, pj, pk).
__global__ void grad_physical_kernel(const double *__restrict__ g64, Dims d, int nx, int ny, int nz,
                                     int nb, double scale, double *__restrict__ out) {
  const size_t n = (size_t)nx * ny * nz;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x) {
    const int pi = (int)(q % nx);
    const size_t rest = q / nx;
    const int pj = (int)(rest % ny), pk = (int)(rest / ny);
    const int i0 = pi == 0 ? 0 : pi + nb, i1 = pi == nx - 1 ? d.NX - 1 : pi + nb;
    const int j0 = pj == 0 ? 0 : pj + nb, j1 = pj == ny - 1 ? d.NY - 1 : pj + nb;
    const int k0 = pk == 0 ? 0 : pk + nb, k1 = pk == nz - 1 ? d.NZ - 1 : pk + nb;
    double s = 0.0;
    for (int k = k0; k <= k1; ++k)
      for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) s += g64[((size_t)k * d.NY + j) * d.Xp + i];
    out[q] = scale * s;
  }
}

static int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

static int row_grid(const Dims &d) {
  const long r = (long)d.NY * d.NZ;
  return (int)(r < 152 * 64 ? (r < 1 ? 1 : r) : 152 * 64);
}

cudaError_t launch_grad_accum(int storage, const void *mu, const void *u1, const void *u0,
                              const void *um1, float *g32, Dims d, Sponge sp, cudaStream_t st) {
  const size_t nq = d.vol() / 4;
  if (d.Xp % 4 == 0 && nq < 0x7fffffffull) {
    const int blocks = grid_for(nq);
    switch (storage) {
      case FDW_F32:
        grad_accum4_kernel<float><<<blocks, 256, 0, st>>>((const float *)mu, (const float *)u1, (const float *)u0,
                                                          (const float *)um1, g32, d, sp, (int)nq);
        break;
      case FDW_BF16:
        grad_accum4_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(
            (const __nv_bfloat16 *)mu, (const __nv_bfloat16 *)u1, (const __nv_bfloat16 *)u0,
            (const __nv_bfloat16 *)um1, g32, d, sp, (int)nq);
        break;
      case FDW_F16:
        grad_accum4_kernel<__half><<<blocks, 256, 0, st>>>((const __half *)mu, (const __half *)u1,
                                                           (const __half *)u0, (const __half *)um1, g32, d, sp,
                                                           (int)nq);
        break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (storage) {
    case FDW_F32:
      grad_accum_kernel<float><<<row_grid(d), 256, 0, st>>>(
          (const float *)mu, (const float *)u1, (const float *)u0, (const float *)um1, g32, d, sp);
      break;
    case FDW_BF16:
      grad_accum_kernel<__nv_bfloat16><<<row_grid(d), 256, 0, st>>>(
          (const __nv_bfloat16 *)mu, (const __nv_bfloat16 *)u1, (const __nv_bfloat16 *)u0,
          (const __nv_bfloat16 *)um1, g32, d, sp);
      break;
    case FDW_F16:
      grad_accum_kernel<__half><<<row_grid(d), 256, 0, st>>>(
          (const __half *)mu, (const __half *)u1, (const __half *)u0, (const __half *)um1, g32, d, sp);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_accum_pair(int storage, const void *mu_a, const void *mu_b, const void *ua,
                                   const void *ub, const void *uc, const void *ud, float *g32, Dims d, Sponge sp,
                                   cudaStream_t st) {
  const size_t nq = d.vol() / 4;
  if (d.Xp % 4 != 0 || nq >= 0x7fffffffull) {  // two single terms
    cudaError_t e = launch_grad_accum(storage, mu_a, ua, ub, uc, g32, d, sp, st);
    return e != cudaSuccess ? e : launch_grad_accum(storage, mu_b, ub, uc, ud, g32, d, sp, st);
  }
  const int blocks = grid_for(nq);
  switch (storage) {
    case FDW_F32:
      grad_accum4_pair_kernel<float><<<blocks, 256, 0, st>>>(
          (const float *)mu_a, (const float *)mu_b, (const float *)ua, (const float *)ub, (const float *)uc,
          (const float *)ud, g32, d, sp, (int)nq);
      break;
    case FDW_BF16:
      grad_accum4_pair_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(
          (const __nv_bfloat16 *)mu_a, (const __nv_bfloat16 *)mu_b, (const __nv_bfloat16 *)ua,
          (const __nv_bfloat16 *)ub, (const __nv_bfloat16 *)uc, (const __nv_bfloat16 *)ud, g32, d, sp, (int)nq);
      break;
    case FDW_F16:
      grad_accum4_pair_kernel<__half><<<blocks, 256, 0, st>>>(
          (const __half *)mu_a, (const __half *)mu_b, (const __half *)ua, (const __half *)ub, (const __half *)uc,
          (const __half *)ud, g32, d, sp, (int)nq);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_flush(float *g32, double *g64, size_t n, cudaStream_t st) {
  grad_flush_kernel<<<grid_for(n), 256, 0, st>>>(g32, g64, n);
  return cudaGetLastError();
}

cudaError_t launch_grad_physical(const double *g64, Dims d, int nx, int ny, int nz, int nb,
                                 double scale, double *out, cudaStream_t st) {
  grad_physical_kernel<<<grid_for((size_t)nx * ny * nz), 256, 0, st>>>(g64, d, nx, ny, nz, nb,
                                                                       scale, out);
  return cudaGetLastError();
}

}  // namespace fdw
