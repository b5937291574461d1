// sparse.cu -- per-step sparse work after the stencil update:
//   * source injection ("Add Source" of Algorithm 1): each point source is a
//     discrete delta, trilinear weight / h^3, scaled like the stencil term,
//     u+ += c w amp / (h^3 P) with c = dt^2 v^2. With the stored coefficient
//     c' = (v dt / h)^2 this is c' w amp / (h P);
//   * receiver interpolation: trace[n+1][rec] = sum_corner w u+(corner),
//     FP32 values, FP64 products, sum and storage.
// The injection kernel is also the step counter: it reads n, publishes n+1.
#include "fdw_internal.h"
#include "fdwave.h"

namespace fdw {

template <typename T> __device__ __forceinline__ void atomic_add_st(T *p, float v);
template <> __device__ __forceinline__ void atomic_add_st<float>(float *p, float v) {
  atomicAdd(p, v);
}
template <> __device__ __forceinline__ void atomic_add_st<__nv_bfloat16>(__nv_bfloat16 *p, float v) {
  atomicAdd(p, __float2bfloat16_rn(v));
}
template <> __device__ __forceinline__ void atomic_add_st<__half>(__half *p, float v) {
  atomicAdd(p, __float2half_rn(v));
}

// Corner layout shared by sources and receivers: for point s and corner q,
// ijk[(s*8+q)*3 + a] are the computational-grid indices (always inside the
// grid; dropped corners have weight 0).
// Forward injection of step n by the threads of one block.
template <typename T>
__device__ __forceinline__ void inject_step(const SparseLaunch &L, int n, size_t plane) {
  for (int t = threadIdx.x; t < L.nsrc * 8; t += blockDim.x) {
    const float wt = L.src_w[t];
    if (wt == 0.f) continue;
    const int s = t >> 3;
    const int i = L.src_corner[t * 3 + 0], j = L.src_corner[t * 3 + 1], k = L.src_corner[t * 3 + 2];
    const size_t p = (size_t)k * plane + (size_t)j * L.d.Xp + i;
    const float amp = L.wavelet[(size_t)n * L.nsrc + s];
    const float gh = L.sp.gx[i] + L.sp.gy[j] + L.sp.gz[k];
    const float cc = St<T>::ld(((const T *)L.c)[p]);
    const float v = cc * wt * (amp * L.amp_scale) * __frcp_rn(1.f + gh);
    atomic_add_st<T>((T *)L.f0 + p, v);
    if (L.f1) atomic_add_st<T>((T *)L.f1 + p, v);
  }
}

// Receiver r's trace value of level n1.
template <typename T>
__device__ __forceinline__ void gather_receiver(const SparseLaunch &L, int r, int n1, size_t plane) {
  const T *f = (const T *)L.f0;
  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int t = r * 8 + q;
    const float wt = L.rec_w[t];
    const int i = L.rec_corner[t * 3 + 0], j = L.rec_corner[t * 3 + 1], k = L.rec_corner[t * 3 + 2];
    const float v = St<T>::ld(f[(size_t)k * plane + (size_t)j * L.d.Xp + i]);
    acc += (double)wt * (double)v;
  }
  L.traces[(size_t)n1 * L.nrec + r] = acc * L.trace_scale;
}

template <typename T>
__global__ void __launch_bounds__(256) inject_kernel(SparseLaunch L) {
  __shared__ int sn;
  if (threadIdx.x == 0) sn = *L.step;
  __syncthreads();
  const int n = sn;
  if (threadIdx.x == 0) *L.step = L.adjoint ? n - 1 : n + 1;
  const size_t plane = L.d.plane();
  if (!L.adjoint) {
    if (n >= 0 && n < L.nt_src) inject_step<T>(L, n, plane);
  } else {
    // Adjoint step that produced level k = n - 1 (the residual was spread by
    // adjoint_spread_kernel just before). Source side of the adjoint:
    // d J / d wavelet[k-1][s] = sum_corner w / h^3 mu_k (the stored source
    // weights are w / h; src_adj_scale = 1 / h^2).
    const int k = n - 1;
    if (k < 0) return;
    if (L.src_adj && k >= 1 && k - 1 < L.nt_src) {
      for (int s = threadIdx.x; s < L.nsrc; s += blockDim.x) {
        double acc = 0.0;
        for (int q = 0; q < 8; ++q) {
          const int t = s * 8 + q;
          const int i = L.src_corner[t * 3 + 0], j = L.src_corner[t * 3 + 1], kk = L.src_corner[t * 3 + 2];
          const float v = St<T>::ld(((const T *)L.f0)[(size_t)kk * plane + (size_t)j * L.d.Xp + i]);
          acc += (double)L.src_w[t] * (double)v;
        }
        L.src_adj[(size_t)(k - 1) * L.nsrc + s] = acc * (double)L.src_adj_scale;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) gather_kernel(SparseLaunch L) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= L.nrec) return;
  const int n1 = *L.step;  // level just produced
  if (n1 < 0 || n1 > L.nt_rec) return;
  gather_receiver<T>(L, r, n1, L.d.plane());
}

// Adjoint step producing level k = *step - 1 (the counter is decremented by
// the injection kernel that follows): spread residual row k with the
// receiver weights (no 1/h^3), scaled like the stencil term,
// dt^2 v^2 w res / P = c' h^2 w res / P. One thread per receiver corner.
template <typename T>
__global__ void __launch_bounds__(256) adjoint_spread_kernel(SparseLaunch L) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.nrec * 8) return;
  const int k = *L.step - 1;
  if (k < 0 || k > L.nt_res) return;
  const float wt = L.rec_w[t];
  if (wt == 0.f) return;
  const int s = t >> 3;
  const int i = L.rec_corner[t * 3 + 0], j = L.rec_corner[t * 3 + 1], kk = L.rec_corner[t * 3 + 2];
  const size_t p = (size_t)kk * L.d.plane() + (size_t)j * L.d.Xp + i;
  const float res = (float)L.residual[(size_t)k * L.nrec + s];
  const float gh = L.sp.gx[i] + L.sp.gy[j] + L.sp.gz[kk];
  const float cc = St<T>::ld(((const T *)L.c)[p]);
  atomic_add_st<T>((T *)L.f0 + p, cc * L.res_scale * wt * (res * L.amp_scale) * __frcp_rn(1.f + gh));
}

// Forward step with at most kFusedRec receivers: injection and receiver
// interpolation in one block (one launch instead of two; the block barrier
// orders the injection's atomics before the receivers' reads). Same
// arithmetic as inject_kernel + gather_kernel.
constexpr int kFusedRec = 256;  // one receiver per thread of the block

template <typename T>
__global__ void __launch_bounds__(256) inject_gather_kernel(SparseLaunch L) {
  __shared__ int sn;
  if (threadIdx.x == 0) sn = *L.step;
  __syncthreads();
  const int n = sn;
  if (threadIdx.x == 0) *L.step = n + 1;
  const size_t plane = L.d.plane();
  if (n >= 0 && n < L.nt_src) inject_step<T>(L, n, plane);
  __syncthreads();
  const int n1 = n + 1;  // level just produced
  const int r = threadIdx.x;
  if (r < L.nrec && n1 >= 0 && n1 <= L.nt_rec) gather_receiver<T>(L, r, n1, plane);
}

template <typename T>
static cudaError_t launch_sparse_t(const SparseLaunch &L, cudaStream_t st) {
  cudaError_t e;
  if (!L.adjoint && L.nrec > 0 && L.nrec <= kFusedRec && L.traces) {
    inject_gather_kernel<T><<<1, 256, 0, st>>>(L);
    return cudaGetLastError();
  }
  if (L.adjoint && L.residual && L.nrec > 0) {
    adjoint_spread_kernel<T><<<(L.nrec * 8 + 255) / 256, 256, 0, st>>>(L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  inject_kernel<T><<<1, 256, 0, st>>>(L);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!L.adjoint && L.nrec > 0 && L.traces) {
    gather_kernel<T><<<(L.nrec + 255) / 256, 256, 0, st>>>(L);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_sparse(const SparseLaunch &L, cudaStream_t st) {
  switch (L.storage) {
    case FDW_F32: return launch_sparse_t<float>(L, st);
    case FDW_BF16: return launch_sparse_t<__nv_bfloat16>(L, st);
    case FDW_F16: return launch_sparse_t<__half>(L, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fdw
