// misfit.cu -- FWI data misfit: residual r = d - d_obs and
// J = 1/2 sum r^2 in FP64 (the objective whose gradient fdw_adjoint_* gives).
//
// Deterministic two-pass reduction: block b owns the fixed chunk
// [b kMisfitChunk, (b+1) kMisfitChunk) and writes its partial sum to a
// scratch array; one block then adds the partials in a fixed order. The
// result does not depend on the launch or on other work on the GPU.
#include <stdint.h>

#include <mutex>

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

// dJ/dv = dJ/dm dm/dv with m = 1/v^2: -2 v^-3 dJ/dm, elementwise in FP64.
__global__ void __launch_bounds__(256)
    velocity_gradient_kernel(const float *__restrict__ v, const double *__restrict__ gm, long long n,
                             double *__restrict__ gv) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double vi = (double)v[i];
    gv[i] = -2.0 * gm[i] / (vi * vi * vi);
  }
}

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

// ---------------------------------------------------------------------------
// Allocation-free variant. Its chunk sums live in this file-scope device
// array (256 KB on every GPU that loads the library, kept until the process
// exits) instead of memory taken per call. Host code cannot use the
// array's name as a device address: the address is looked up once per
// device with cudaGetSymbolAddress and cached below.
// ---------------------------------------------------------------------------
namespace {
constexpr long long kNoAllocChunks = 32768;
constexpr long long kNoAllocMaxValues = kNoAllocChunks * fdw::kMisfitChunk;  // 67,108,864
static __device__ __align__(256) double g_misfit_scratch[kNoAllocChunks];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double *g_scratch_addr[kMaxDevices] = {};
}  // namespace

extern "C" int fdw_misfit_noalloc(const double *d, const double *d_obs, long long n,
                                  double *residual, double *J, void *stream) {
  if ((n > 0 && (!d || !d_obs)) || !J || n < 0)
    return report_error(FDW_ERR_INVALID_ARG, "fdw_misfit_noalloc: NULL pointer or n < 0");
  if (n > kNoAllocMaxValues)
    return report_error(FDW_ERR_INVALID_ARG,
                        "fdw_misfit_noalloc: n = %lld exceeds the maximum of %lld values "
                        "(static scratch of %lld chunk sums); use fdw_misfit",
                        n, kNoAllocMaxValues, kNoAllocChunks);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return report_error(FDW_ERR_CUDA, "fdw_misfit_noalloc: no usable current device");
  }
  double *scratch;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      // set-up, once per device, with that device current
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_misfit_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return report_error(FDW_ERR_CUDA, "fdw_misfit_noalloc: cudaGetSymbolAddress: %s",
                            cudaGetErrorString(e));
      }
      g_scratch_addr[dev] = (double *)p;
    }
    scratch = g_scratch_addr[dev];
  }
  e = launch_misfit(d, d_obs, n, residual, J, scratch, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return report_error(FDW_ERR_CUDA, "fdw_misfit_noalloc: %s", cudaGetErrorString(e));
  }
  return FDW_OK;
}

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

extern "C" int fdw_velocity_gradient(const float *vp, const double *grad_m, long long n, double *grad_v,
                                     void *stream) {
  if (n < 0 || (n > 0 && (!vp || !grad_m || !grad_v)))
    return report_error(FDW_ERR_INVALID_ARG, "fdw_velocity_gradient: NULL pointer or n < 0");
  if (n == 0) return FDW_OK;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  velocity_gradient_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(vp, grad_m, n, grad_v);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report_error(FDW_ERR_CUDA, "fdw_velocity_gradient: %s", cudaGetErrorString(e));
  return FDW_OK;
}
