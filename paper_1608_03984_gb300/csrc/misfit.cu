// misfit.cu -- FWI data misfit: residual r = d - d_obs and
// J = 1/2 sum r^2 in FP64 (the objective whose gradient fdw_adjoint_* gives).
//
// Deterministic two-pass reduction: block b owns the fixed chunk
// [b kMisfitChunk, (b+1) kMisfitChunk) and writes its partial sum to a
// scratch array; one block then adds the partials in a fixed order. The
// result does not depend on the launch or on other work on the GPU.
#include <stdint.h>

#include "fdw_internal.h"
#include "fdwave.h"

namespace fdw {

constexpr int kMisfitThreads = 256;
constexpr int kMisfitChunk = kMisfitThreads * 8;  // elements per partial sum

__global__ void __launch_bounds__(kMisfitThreads)
    misfit_partial_kernel(const double *__restrict__ d, const double *__restrict__ o, long long n,
                          double *__restrict__ res, double *__restrict__ partial) {
  __shared__ double red[kMisfitThreads];
  const long long base = (long long)blockIdx.x * kMisfitChunk;
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kMisfitChunk / kMisfitThreads; ++i) {
    const long long p = base + (long long)i * kMisfitThreads + threadIdx.x;
    if (p < n) {
      const double r = d[p] - o[p];
      if (res) res[p] = r;
      s = fma(r, r, s);
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kMisfitThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kMisfitThreads)
    misfit_final_kernel(const double *__restrict__ partial, long long nchunks, double *__restrict__ J) {
  __shared__ double red[kMisfitThreads];
  double s = 0.0;
  for (long long c = threadIdx.x; c < nchunks; c += kMisfitThreads) s += partial[c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kMisfitThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *J = 0.5 * red[0];
}

long long misfit_chunks(long long n) { return (n + kMisfitChunk - 1) / kMisfitChunk; }

cudaError_t launch_misfit(const double *d, const double *o, long long n, double *res, double *J,
                          double *partial, cudaStream_t st) {
  const long long nc = misfit_chunks(n);
  if (nc > 0) {
    if (nc > 0x7fffffffLL) return cudaErrorInvalidValue;
    misfit_partial_kernel<<<(unsigned)nc, kMisfitThreads, 0, st>>>(d, o, n, res, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  misfit_final_kernel<<<1, kMisfitThreads, 0, st>>>(partial, nc, J);
  return cudaGetLastError();
}

}  // namespace fdw

using namespace fdw;

extern "C" int fdw_misfit(const double *d, const double *d_obs, long long n, double *residual,
                          double *J, void *stream) {
  if ((n > 0 && (!d || !d_obs)) || !J || n < 0)
    return report_error(FDW_ERR_INVALID_ARG, "fdw_misfit: NULL pointer or n < 0");
  cudaStream_t st = (cudaStream_t)stream;
  const long long nc = misfit_chunks(n);
  double *partial = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&partial, (size_t)(nc > 0 ? nc : 1) * sizeof(double), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return report_error(e == cudaErrorMemoryAllocation ? FDW_ERR_OOM : FDW_ERR_CUDA,
                        "fdw_misfit: scratch allocation: %s", cudaGetErrorString(e));
  }
  e = launch_misfit(d, d_obs, n, residual, J, partial, st);
  cudaError_t e2 = cudaFreeAsync(partial, st);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    return report_error(FDW_ERR_CUDA, "fdw_misfit: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  return FDW_OK;
}
