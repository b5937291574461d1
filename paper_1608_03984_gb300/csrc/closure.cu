// closure.cu -- the learned closure: a 3x3x3 convolutional network
// (3 -> 16 -> 16 -> 1 channels, ReLU between) that corrects a coarse,
// low-order time step toward the fine, high-order one. The paper has no
// learned component; its cost-benefit section (coarse grid with a high
// order vs fine grid with a low order) is the trade-off this closure works
// on. Weights are stored in BF16, every sum is accumulated in FP32.
//
// Training works on batches of cubic patches (valid convolutions: an input
// patch of S points per axis gives S-6 outputs); inference runs on a whole
// computational grid inside the time loop ("same" convolutions, zero
// outside the grid), normalised by the largest |u_n| of the current level:
//   x = (u_n / s, u_{n-1} / s, (v - 3000) / 750),
//   u_{n+1} += s * (net(x) - net(x0)),  x0 = (0, 0, (v - 3000) / 750).
// Subtracting the network's answer for a zero wavefield makes the
// correction vanish where the wave has not arrived: any output there would
// be integrated twice by the leapfrog update and grow quadratically in time.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "fdw_internal.h"
#include "fdwave.h"

namespace fdw {

constexpr int kH = 16;  // hidden channels
constexpr int kOffW1 = 0, kOffB1 = kH * 3 * 27, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH * 27,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * 27, kNumParams = kOffB3 + 1;
constexpr float kVelMean = 3000.f, kVelScale = 750.f;
constexpr int kBwdChunks = 16;  // partial sums per weight-gradient pair
constexpr int kHalo = kClosureHalo;  // receptive-field radius of the three 3x3x3 layers

// ---------------------------------------------------------------------------
// convolutions
// ---------------------------------------------------------------------------
// Geometry of one convolution: input box (zi, yi, xi) per sample and
// channel, output box (zo, yo, xo); input index = output index + tap - off
// (off = 0: valid, off = 1: same with zero outside the input box).
struct ConvGeom {
  int B, zi, yi, xi, zo, yo, xo, off;
  __host__ __device__ long long in_vol() const { return (long long)zi * yi * xi; }
  __host__ __device__ long long out_vol() const { return (long long)zo * yo * xo; }
};

// (x, y, z, b) of a linear index over [B][zd][yd][xd]; 32-bit division
// when the index fits (every use here), 64-bit otherwise.
__device__ __forceinline__ void split_index(long long q, int xd, int yd, int zd, int &x, int &y, int &z,
                                            int &b) {
  if (q <= 0x7fffffffLL) {
    unsigned u = (unsigned)q;
    x = (int)(u % (unsigned)xd);
    u /= (unsigned)xd;
    y = (int)(u % (unsigned)yd);
    u /= (unsigned)yd;
    z = (int)(u % (unsigned)zd);
    b = (int)(u / (unsigned)zd);
  } else {
    x = (int)(q % xd);
    long long r = q / xd;
    y = (int)(r % yd);
    r /= yd;
    z = (int)(r % zd);
    b = (int)(r / zd);
  }
}

template <int CI, int CO, bool RELU>
__global__ void __launch_bounds__(256)
    conv_fwd_kernel(const float *__restrict__ in, const __nv_bfloat16 *__restrict__ w,
                    const float *__restrict__ bias, float *__restrict__ out, ConvGeom g) {
  __shared__ float ws[CO * CI * 27];
  for (int i = threadIdx.x; i < CO * CI * 27; i += blockDim.x) ws[i] = __bfloat162float(w[i]);
  __syncthreads();
  const long long nout = (long long)g.B * g.out_vol();
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nout;
       q += (long long)gridDim.x * blockDim.x) {
    int x, y, z, b;
    split_index(q, g.xo, g.yo, g.zo, x, y, z, b);
    float acc[CO];
#pragma unroll
    for (int o = 0; o < CO; ++o) acc[o] = bias[o];
    const float *inb = in + (long long)b * CI * g.in_vol();
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
      const int zz = z + a - g.off;
      if (zz < 0 || zz >= g.zi) continue;
#pragma unroll 1
      for (int bb = 0; bb < 3; ++bb) {
        const int yy = y + bb - g.off;
        if (yy < 0 || yy >= g.yi) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int xx = x + c - g.off;
          if (xx < 0 || xx >= g.xi) continue;
          const int tap = (a * 3 + bb) * 3 + c;
          const long long p = ((long long)zz * g.yi + yy) * g.xi + xx;
#pragma unroll
          for (int i = 0; i < CI; ++i) {
            const float v = inb[(long long)i * g.in_vol() + p];
#pragma unroll
            for (int o = 0; o < CO; ++o) acc[o] = fmaf(ws[(o * CI + i) * 27 + tap], v, acc[o]);
          }
        }
      }
    }
    float *outb = out + (long long)b * CO * g.out_vol() + ((long long)z * g.yo + y) * g.xo + x;
#pragma unroll
    for (int o = 0; o < CO; ++o) outb[(long long)o * g.out_vol()] = RELU ? fmaxf(acc[o], 0.f) : acc[o];
  }
}

// d loss / d input of a convolution (valid geometry: input = output + tap),
// masked by the ReLU of the input activation when `act` is given.
template <int CI, int CO>
__global__ void __launch_bounds__(256)
    conv_bwd_data_kernel(const float *__restrict__ gout, const __nv_bfloat16 *__restrict__ w,
                         const float *__restrict__ act, float *__restrict__ gin, ConvGeom g) {
  __shared__ float ws[CO * CI * 27];
  for (int i = threadIdx.x; i < CO * CI * 27; i += blockDim.x) ws[i] = __bfloat162float(w[i]);
  __syncthreads();
  const long long nin = (long long)g.B * g.in_vol();
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nin;
       q += (long long)gridDim.x * blockDim.x) {
    int x, y, z, b;
    split_index(q, g.xi, g.yi, g.zi, x, y, z, b);
    float acc[CI];
#pragma unroll
    for (int i = 0; i < CI; ++i) acc[i] = 0.f;
    const float *gb = gout + (long long)b * CO * g.out_vol();
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
      const int zo = z - a;
      if (zo < 0 || zo >= g.zo) continue;
#pragma unroll 1
      for (int bb = 0; bb < 3; ++bb) {
        const int yo = y - bb;
        if (yo < 0 || yo >= g.yo) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int xo = x - c;
          if (xo < 0 || xo >= g.xo) continue;
          const int tap = (a * 3 + bb) * 3 + c;
          const long long p = ((long long)zo * g.yo + yo) * g.xo + xo;
#pragma unroll
          for (int o = 0; o < CO; ++o) {
            const float gv = gb[(long long)o * g.out_vol() + p];
#pragma unroll
            for (int i = 0; i < CI; ++i) acc[i] = fmaf(ws[(o * CI + i) * 27 + tap], gv, acc[i]);
          }
        }
      }
    }
    const long long base = (long long)b * CI * g.in_vol() + ((long long)z * g.yi + y) * g.xi + x;
#pragma unroll
    for (int i = 0; i < CI; ++i) {
      const long long p = base + (long long)i * g.in_vol();
      gin[p] = (act && act[p] <= 0.f) ? 0.f : acc[i];
    }
  }
}

// Weight/bias gradient, stage 1: block (pair = o*CI + i, chunk) sums over its
// share of the (sample, output point) pairs the 27 products in * gout and,
// for i == 0, gout itself (the bias term); writes 28 partial sums.
template <int CI, int CO>
__global__ void __launch_bounds__(256)
    conv_bwd_weight_kernel(const float *__restrict__ in, const float *__restrict__ gout,
                           float *__restrict__ partial, ConvGeom g) {
  const int pair = blockIdx.x, chunk = blockIdx.y;
  const int o = pair / CI, i = pair % CI;
  float acc[28];
#pragma unroll
  for (int t = 0; t < 28; ++t) acc[t] = 0.f;
  const long long nout = (long long)g.B * g.out_vol();
  const long long per = (nout + gridDim.y - 1) / gridDim.y;
  const long long q0 = (long long)chunk * per, q1 = q0 + per < nout ? q0 + per : nout;
  for (long long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    int x, y, z, b;
    split_index(q, g.xo, g.yo, g.zo, x, y, z, b);
    const float gv = gout[((long long)b * CO + o) * g.out_vol() + ((long long)z * g.yo + y) * g.xo + x];
    const float *inb = in + ((long long)b * CI + i) * g.in_vol();
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          acc[(a * 3 + bb) * 3 + c] =
              fmaf(gv, inb[((long long)(z + a) * g.yi + (y + bb)) * g.xi + (x + c)], acc[(a * 3 + bb) * 3 + c]);
    acc[27] += gv;
  }
  __shared__ float red[256];
  for (int t = 0; t < 28; ++t) {
    red[threadIdx.x] = acc[t];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[((long long)pair * gridDim.y + chunk) * 28 + t] = red[0];
    __syncthreads();
  }
}

// Stage 2: add the chunk partials in order into the gradient vector.
template <int CI, int CO>
__global__ void conv_bwd_weight_reduce(const float *__restrict__ partial, int chunks,
                                       float *__restrict__ gw, float *__restrict__ gbias) {
  const int pair = blockIdx.x, t = threadIdx.x;
  if (t >= 28) return;
  float s = 0.f;
  for (int c = 0; c < chunks; ++c) s += partial[((long long)pair * chunks + c) * 28 + t];
  const int o = pair / CI, i = pair % CI;
  if (t < 27) gw[(o * CI + i) * 27 + t] = s;
  else if (i == 0) gbias[o] = s;
}

// Paired MSE: out holds net(x) for B samples then net(x0) for the same B;
// r = out[q] - out[q + n] - t[q]; gradient 2 r / M into the first half and
// -2 r / M into the second; per-block partial sums of r^2 / M.
__global__ void mse_pair_kernel(const float *__restrict__ out, const float *__restrict__ t, long long n,
                                float inv_m, float *__restrict__ g, float *__restrict__ partial) {
  __shared__ float red[256];
  float s = 0.f;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const float r = out[q] - out[q + n] - t[q];
    if (g) {
      g[q] = 2.f * r * inv_m;
      g[q + n] = -2.f * r * inv_m;
    }
    s = fmaf(r * r, inv_m, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// xpair = [x ; x with the two wavefield channels zeroed]: [2B][3][S^3].
__global__ void pair_batch_kernel(const float *__restrict__ x, long long B, long long s3,
                                  float *__restrict__ xpair) {
  const long long n = B * 3 * s3;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const float v = x[q];
    xpair[q] = v;
    xpair[n + q] = (q / s3) % 3 == 2 ? v : 0.f;
  }
}

// out = net(x) - net(x0) from the paired output [2B][n3 per sample].
__global__ void pair_diff_kernel(const float *__restrict__ pout, long long n, float *__restrict__ out) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    out[q] = pout[q] - pout[q + n];
}

__global__ void sum_partials_kernel(const float *__restrict__ partial, int n, float *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += partial[i];
    *out = s;
  }
}

// Adam on the FP32 master parameters; refreshes the BF16 copy. The
// constants 1 - beta and the bias corrections 1 - beta^t come from the host
// in FP64 (in FP32, 1 - 0.999 would already be off by 1e-5 relative).
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ pb, int n, float lr,
                            float b1, float omb1, float b2, float omb2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + omb1 * gi;
  const float vi = b2 * v[i] + omb2 * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  pb[i] = __float2bfloat16_rn(pi);
}

__global__ void to_bf16_kernel(const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

// ---------------------------------------------------------------------------
// inference inside the time loop
// ---------------------------------------------------------------------------
// s = max |u_n| over the computational grid (a bound independent of the
// grid's size, so a net trained on small boxes sees the same input scale on
// large ones): per-block maxima, then one block. Max is order-independent,
// so s is deterministic.
template <typename T>
__global__ void absmax_partial_kernel(const T *__restrict__ u, Dims d, float *__restrict__ partial) {
  __shared__ float red[256];
  float s = 0.f;
  const size_t n = d.vol();
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n;
       p += (size_t)gridDim.x * blockDim.x)
    s = fmaxf(s, fabsf(St<T>::ld(u[p])));  // padding columns hold 0
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void absmax_final_kernel(const float *__restrict__ partial, int n, float *__restrict__ s_out) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fmaxf(s, partial[i]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *s_out = red[0] > 1e-30f ? red[0] : 1e-30f;
}

// x[0] = u_n / s, x[1] = u_{n-1} / s, x[2] = (v - 3000) / 750, dense
// [3][NZ][NY][NX]; v from the physical model, extended into the sponge.
template <typename T>
__global__ void closure_inputs_kernel(const T *__restrict__ u, const T *__restrict__ um,
                                      const float *__restrict__ vp, int nx, int ny, int nz, int nb,
                                      Dims d, const float *__restrict__ s_dev, float *__restrict__ x) {
  const float inv = u ? 1.f / *s_dev : 0.f;  // u == null: the zero-wavefield input x0
  const long long n = (long long)d.NX * d.NY * d.NZ;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % d.NX);
    const long long r = q / d.NX;
    const int j = (int)(r % d.NY), k = (int)(r / d.NY);
    const size_t p = ((size_t)k * d.NY + j) * d.Xp + i;
    const int pi = min(max(i - nb, 0), nx - 1), pj = min(max(j - nb, 0), ny - 1),
              pk = min(max(k - nb, 0), nz - 1);
    x[q] = u ? St<T>::ld(u[p]) * inv : 0.f;
    x[n + q] = u ? St<T>::ld(um[p]) * inv : 0.f;
    x[2 * n + q] = (vp[((size_t)pk * ny + pj) * nx + pi] - kVelMean) / kVelScale;
  }
}

// Last layer fused with the update: u_{n+1} += s * (b3 + sum W3 a2 - base)
// on the physical points whose 7^3 receptive field is physical too:
// [nb + 3, nb + n - 3) along each axis. The sponge and the 3 points next
// to it keep the plain update: the sponge's job is absorption, which the
// fine solver does not define on the coarse grid.
template <typename T>
__global__ void __launch_bounds__(256)
    closure_apply_kernel(const float *__restrict__ a2, const __nv_bfloat16 *__restrict__ w3,
                         const float *__restrict__ b3, const float *__restrict__ base,
                         const float *__restrict__ s_dev, T *__restrict__ u, Dims d, int nb, int nx,
                         int ny, int nz, float factor) {
  __shared__ float ws[kH * 27];
  for (int i = threadIdx.x; i < kH * 27; i += blockDim.x) ws[i] = __bfloat162float(w3[i]);
  __syncthreads();
  const float s = factor * *s_dev;
  const long long vol = (long long)d.NX * d.NY * d.NZ;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < vol;
       q += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(q % d.NX);
    const long long r = q / d.NX;
    const int y = (int)(r % d.NY), z = (int)(r / d.NY);
    if (x < nb + kHalo || x >= nb + nx - kHalo || y < nb + kHalo || y >= nb + ny - kHalo ||
        z < nb + kHalo || z >= nb + nz - kHalo)
      continue;
    float acc = b3[0];
    for (int a = 0; a < 3; ++a) {
      const int zz = z + a - 1;
      if (zz < 0 || zz >= d.NZ) continue;
      for (int bb = 0; bb < 3; ++bb) {
        const int yy = y + bb - 1;
        if (yy < 0 || yy >= d.NY) continue;
        for (int c = 0; c < 3; ++c) {
          const int xx = x + c - 1;
          if (xx < 0 || xx >= d.NX) continue;
          const long long p = ((long long)zz * d.NY + yy) * d.NX + xx;
          const int tap = (a * 3 + bb) * 3 + c;
#pragma unroll
          for (int i = 0; i < kH; ++i) acc = fmaf(ws[i * 27 + tap], a2[(long long)i * vol + p], acc);
        }
      }
    }
    acc -= base[q];
    const size_t pp = ((size_t)z * d.NY + y) * d.Xp + x;
    u[pp] = St<T>::st(St<T>::ld(u[pp]) + s * acc);
  }
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t closure_forward_batch(const float *x, const __nv_bfloat16 *pb, const float *pf, int B,
                                  int S, float *a1, float *a2, float *out, cudaStream_t st) {
  ConvGeom g1{B, S, S, S, S - 2, S - 2, S - 2, 0};
  ConvGeom g2{B, S - 2, S - 2, S - 2, S - 4, S - 4, S - 4, 0};
  ConvGeom g3{B, S - 4, S - 4, S - 4, S - 6, S - 6, S - 6, 0};
  conv_fwd_kernel<3, kH, true><<<grid_for(B * g1.out_vol()), 256, 0, st>>>(x, pb + kOffW1, pf + kOffB1, a1, g1);
  conv_fwd_kernel<kH, kH, true><<<grid_for(B * g2.out_vol()), 256, 0, st>>>(a1, pb + kOffW2, pf + kOffB2, a2, g2);
  conv_fwd_kernel<kH, 1, false><<<grid_for(B * g3.out_vol()), 256, 0, st>>>(a2, pb + kOffW3, pf + kOffB3, out, g3);
  return cudaGetLastError();
}

// Inference workspace for one grid: the FP32 path keeps the inputs and both
// hidden layers on the whole grid (35 floats per point), the tensor-core
// path only its FP16 inputs and the network output (closure_tc.cu); both
// keep net(x0) and the normalisation.
int closure_reserve_infer(ClosureNet *c, Dims d) {
  const size_t vol = (size_t)d.NX * d.NY * d.NZ;
  if (c->infer_cap < vol) {
    cudaFree(c->x); cudaFree(c->ia1); cudaFree(c->ia2); cudaFree(c->base);
    c->x = c->ia1 = c->ia2 = c->base = nullptr;
    c->infer_cap = 0;
    if (cudaMalloc(&c->base, vol * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    c->infer_cap = vol;
  }
  if (!c->s_dev && cudaMalloc(&c->s_dev, sizeof(float)) != cudaSuccess) return -1;
  if (!c->s_partial && cudaMalloc(&c->s_partial, 1024 * sizeof(float)) != cudaSuccess) return -1;
  if (c->variant != 1) return closure_tc_reserve(c, d);
  if (!c->x) {
    if (cudaMalloc(&c->x, 3 * vol * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&c->ia1, (size_t)kH * vol * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&c->ia2, (size_t)kH * vol * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(c->x); cudaFree(c->ia1); cudaFree(c->ia2);
      c->x = c->ia1 = c->ia2 = nullptr;
      return -1;
    }
  }
  return 0;
}

template <typename T>
static cudaError_t infer_pre_t(ClosureNet *c, const T *u, const T *um, const float *vp, int nx, int ny,
                               int nz, int nb, Dims d, cudaStream_t st) {
  absmax_partial_kernel<T><<<1024, 256, 0, st>>>(u, d, c->s_partial);
  absmax_final_kernel<<<1, 256, 0, st>>>(c->s_partial, 1024, c->s_dev);
  const long long vol = (long long)d.NX * d.NY * d.NZ;
  closure_inputs_kernel<T><<<grid_for(vol), 256, 0, st>>>(u, um, vp, nx, ny, nz, nb, d, c->s_dev, c->x);
  const ConvGeom g{1, d.NZ, d.NY, d.NX, d.NZ, d.NY, d.NX, 1};
  conv_fwd_kernel<3, kH, true><<<grid_for(vol), 256, 0, st>>>(c->x, c->pb + kOffW1, c->pf + kOffB1, c->ia1, g);
  conv_fwd_kernel<kH, kH, true><<<grid_for(vol), 256, 0, st>>>(c->ia1, c->pb + kOffW2, c->pf + kOffB2, c->ia2, g);
  return cudaGetLastError();
}

cudaError_t closure_infer_base(ClosureNet *c, const float *vp, int nx, int ny, int nz, int nb, Dims d,
                               int *err, cudaStream_t st) {
  if (c->variant != 1) return closure_tc_base(c, vp, nx, ny, nz, nb, d, err, st);
  const long long vol = (long long)d.NX * d.NY * d.NZ;
  closure_inputs_kernel<float><<<grid_for(vol), 256, 0, st>>>(nullptr, nullptr, vp, nx, ny, nz, nb, d, c->s_dev,
                                                              c->x);
  const ConvGeom g{1, d.NZ, d.NY, d.NX, d.NZ, d.NY, d.NX, 1};
  conv_fwd_kernel<3, kH, true><<<grid_for(vol), 256, 0, st>>>(c->x, c->pb + kOffW1, c->pf + kOffB1, c->ia1, g);
  conv_fwd_kernel<kH, kH, true><<<grid_for(vol), 256, 0, st>>>(c->ia1, c->pb + kOffW2, c->pf + kOffB2, c->ia2, g);
  conv_fwd_kernel<kH, 1, false><<<grid_for(vol), 256, 0, st>>>(c->ia2, c->pb + kOffW3, c->pf + kOffB3, c->base, g);
  return cudaGetLastError();
}

template <typename T>
static void absmax_t(ClosureNet *c, const T *u, Dims d, cudaStream_t st) {
  absmax_partial_kernel<T><<<1024, 256, 0, st>>>(u, d, c->s_partial);
  absmax_final_kernel<<<1, 256, 0, st>>>(c->s_partial, 1024, c->s_dev);
}

cudaError_t closure_infer_pre(ClosureNet *c, int storage, const void *u, const void *um, const float *vp,
                              int nx, int ny, int nz, int nb, Dims d, int *err, cudaStream_t st) {
  if (c->variant != 1) {
    switch (storage) {
      case FDW_F32: absmax_t(c, (const float *)u, d, st); break;
      case FDW_BF16: absmax_t(c, (const __nv_bfloat16 *)u, d, st); break;
      case FDW_F16: absmax_t(c, (const __half *)u, d, st); break;
      default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return closure_tc_net(c, storage, u, um, vp, nx, ny, nz, nb, d, err, st);
  }
  switch (storage) {
    case FDW_F32: return infer_pre_t<float>(c, (const float *)u, (const float *)um, vp, nx, ny, nz, nb, d, st);
    case FDW_BF16:
      return infer_pre_t<__nv_bfloat16>(c, (const __nv_bfloat16 *)u, (const __nv_bfloat16 *)um, vp, nx, ny, nz,
                                        nb, d, st);
    case FDW_F16: return infer_pre_t<__half>(c, (const __half *)u, (const __half *)um, vp, nx, ny, nz, nb, d, st);
    default: return cudaErrorInvalidValue;
  }
}

// Tensor-core path: u_{n+1} += s * (net(x) - net(x0)) from the network
// output, on the points whose receptive field is physical.
template <typename T>
__global__ void closure_apply_out_kernel(const float *__restrict__ net, const float *__restrict__ base,
                                         const float *__restrict__ s_dev, T *__restrict__ u, Dims d, int nb,
                                         int nx, int ny, int nz, float factor) {
  const float s = factor * *s_dev;
  // rows (j, k) whose points can be corrected; one block per row
  const int y0 = nb + kHalo, y1 = nb + ny - kHalo, z0 = nb + kHalo, z1 = nb + nz - kHalo;
  const int x0 = nb + kHalo, x1 = nb + nx - kHalo;
  const int ry = y1 - y0, rz = z1 - z0;
  if (ry <= 0 || rz <= 0 || x1 <= x0) return;
  for (int row = blockIdx.x; row < ry * rz; row += gridDim.x) {
    const int y = y0 + row % ry, z = z0 + row / ry;
    const size_t q0 = ((size_t)z * d.NY + y) * d.NX, p0 = ((size_t)z * d.NY + y) * d.Xp;
    for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x)
      u[p0 + x] = St<T>::st(St<T>::ld(u[p0 + x]) + s * (net[q0 + x] - base[q0 + x]));
  }
}

cudaError_t closure_infer_apply(ClosureNet *c, int storage, void *unew, Dims d, int nx, int ny, int nz, int nb,
                                float factor, cudaStream_t st) {
  const long long vol = (long long)d.NX * d.NY * d.NZ;
  if (c->variant != 1) {
    switch (storage) {
      case FDW_F32:
        closure_apply_out_kernel<float><<<grid_for(vol), 256, 0, st>>>(c->tc_out, c->base, c->s_dev, (float *)unew,
                                                                       d, nb, nx, ny, nz, factor);
        break;
      case FDW_BF16:
        closure_apply_out_kernel<__nv_bfloat16><<<grid_for(vol), 256, 0, st>>>(
            c->tc_out, c->base, c->s_dev, (__nv_bfloat16 *)unew, d, nb, nx, ny, nz, factor);
        break;
      case FDW_F16:
        closure_apply_out_kernel<__half><<<grid_for(vol), 256, 0, st>>>(c->tc_out, c->base, c->s_dev,
                                                                        (__half *)unew, d, nb, nx, ny, nz, factor);
        break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (storage) {
    case FDW_F32:
      closure_apply_kernel<float><<<grid_for(vol), 256, 0, st>>>(c->ia2, c->pb + kOffW3, c->pf + kOffB3, c->base, c->s_dev,
                                                                 (float *)unew, d, nb, nx, ny, nz, factor);
      break;
    case FDW_BF16:
      closure_apply_kernel<__nv_bfloat16><<<grid_for(vol), 256, 0, st>>>(
          c->ia2, c->pb + kOffW3, c->pf + kOffB3, c->base, c->s_dev, (__nv_bfloat16 *)unew, d, nb, nx, ny, nz, factor);
      break;
    case FDW_F16:
      closure_apply_kernel<__half><<<grid_for(vol), 256, 0, st>>>(c->ia2, c->pb + kOffW3, c->pf + kOffB3, c->base, c->s_dev,
                                                                  (__half *)unew, d, nb, nx, ny, nz, factor);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t closure_backward_batch(const float *x, const __nv_bfloat16 *pb, int B, int S,
                                   const float *a1, const float *a2, const float *g3, float *g2,
                                   float *g1, float *partial, float *grad, cudaStream_t st) {
  const ConvGeom G1{B, S, S, S, S - 2, S - 2, S - 2, 0};
  const ConvGeom G2{B, S - 2, S - 2, S - 2, S - 4, S - 4, S - 4, 0};
  const ConvGeom G3{B, S - 4, S - 4, S - 4, S - 6, S - 6, S - 6, 0};
  const dim3 wgrid3(kH, kBwdChunks), wgrid2(kH * kH, kBwdChunks), wgrid1(kH * 3, kBwdChunks);
  // layer 3 (16 -> 1)
  conv_bwd_weight_kernel<kH, 1><<<wgrid3, 256, 0, st>>>(a2, g3, partial, G3);
  conv_bwd_weight_reduce<kH, 1><<<kH, 32, 0, st>>>(partial, kBwdChunks, grad + kOffW3, grad + kOffB3);
  conv_bwd_data_kernel<kH, 1><<<grid_for(B * G3.in_vol()), 256, 0, st>>>(g3, pb + kOffW3, a2, g2, G3);
  // layer 2 (16 -> 16)
  conv_bwd_weight_kernel<kH, kH><<<wgrid2, 256, 0, st>>>(a1, g2, partial, G2);
  conv_bwd_weight_reduce<kH, kH><<<kH * kH, 32, 0, st>>>(partial, kBwdChunks, grad + kOffW2, grad + kOffB2);
  conv_bwd_data_kernel<kH, kH><<<grid_for(B * G2.in_vol()), 256, 0, st>>>(g2, pb + kOffW2, a1, g1, G2);
  // layer 1 (3 -> 16)
  conv_bwd_weight_kernel<3, kH><<<wgrid1, 256, 0, st>>>(x, g1, partial, G1);
  conv_bwd_weight_reduce<3, kH><<<kH * 3, 32, 0, st>>>(partial, kBwdChunks, grad + kOffW1, grad + kOffB1);
  return cudaGetLastError();
}

}  // namespace fdw

// ---------------------------------------------------------------------------
// C ABI (include/fdwave.h)
// ---------------------------------------------------------------------------
using namespace fdw;

static void closure_free_train(fdw_closure *c) {
  cudaFree(c->a1); cudaFree(c->a2); cudaFree(c->out); cudaFree(c->g3); cudaFree(c->g2); cudaFree(c->g1);
  c->a1 = c->a2 = c->out = c->g3 = c->g2 = c->g1 = nullptr;
  c->cap1 = c->cap2 = c->cap3 = 0;
}

// Workspace for a batch of B patches of S^3 points, run as 2B samples (each
// patch and its zero-wavefield copy): each layer's buffers grow to the
// largest size asked for so far (patch sizes may change between calls).
static int closure_reserve_train(fdw_closure *c, int B, int S) {
  const size_t B2 = 2 * (size_t)B;
  const size_t s1 = B2 * (S - 2) * (S - 2) * (S - 2), s2 = B2 * (S - 4) * (S - 4) * (S - 4),
               s3 = B2 * (S - 6) * (S - 6) * (S - 6), sx = B2 * 3 * S * S * S;
  if (sx > c->xcap) {
    cudaFree(c->xpair);
    c->xpair = nullptr;
    c->xcap = 0;
    if (cudaMalloc(&c->xpair, sx * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return report_error(FDW_ERR_OOM, "closure: batch of %d patches of %d^3", B, S);
    }
    c->xcap = sx;
  }
  if (s1 <= c->cap1 && s2 <= c->cap2 && s3 <= c->cap3) return FDW_OK;
  const size_t n1 = s1 > c->cap1 ? s1 : c->cap1, n2 = s2 > c->cap2 ? s2 : c->cap2,
               n3 = s3 > c->cap3 ? s3 : c->cap3;
  closure_free_train(c);
  bool ok = cudaMalloc(&c->a1, kH * n1 * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->g1, kH * n1 * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->a2, kH * n2 * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->g2, kH * n2 * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->out, n3 * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->g3, n3 * sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    closure_free_train(c);
    return report_error(FDW_ERR_OOM, "closure: training workspace for %d patches of %d^3", B, S);
  }
  c->cap1 = n1;
  c->cap2 = n2;
  c->cap3 = n3;
  return FDW_OK;
}

// net(x) and net(x0) of a batch: fills c->xpair and c->out ([2B][S-6]^3).
static cudaError_t closure_pair_forward(fdw_closure *c, const float *x, int B, int S) {
  const long long s3 = (long long)S * S * S;
  pair_batch_kernel<<<grid_for(B * 3 * s3), 256, 0, c->stream>>>(x, B, s3, c->xpair);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return closure_forward_batch(c->xpair, c->pb, c->pf, 2 * B, S, c->a1, c->a2, c->out, c->stream);
}

extern "C" long long fdw_closure_num_params(void) { return kNumParams; }

extern "C" int fdw_closure_create(fdw_closure **out, void *stream) {
  if (!out) return report_error(FDW_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  fdw_closure *c = new (std::nothrow) fdw_closure;
  if (!c) return report_error(FDW_ERR_OOM, "host allocation");
  c->stream = (cudaStream_t)stream;
  bool ok = cudaMalloc(&c->pf, kNumParams * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->pb, kNumParams * sizeof(__nv_bfloat16)) == cudaSuccess &&
            cudaMalloc(&c->grad, kNumParams * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->m, kNumParams * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->v, kNumParams * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->partial, (size_t)kH * kH * kBwdChunks * 28 * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->loss_partial, 4096 * sizeof(float)) == cudaSuccess;
  if (ok) {
    ok = cudaMemsetAsync(c->pf, 0, kNumParams * sizeof(float), c->stream) == cudaSuccess &&
         cudaMemsetAsync(c->pb, 0, kNumParams * sizeof(__nv_bfloat16), c->stream) == cudaSuccess &&
         cudaMemsetAsync(c->m, 0, kNumParams * sizeof(float), c->stream) == cudaSuccess &&
         cudaMemsetAsync(c->v, 0, kNumParams * sizeof(float), c->stream) == cudaSuccess &&
         cudaStreamSynchronize(c->stream) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    fdw_closure_destroy(c);
    return report_error(FDW_ERR_OOM, "closure: parameter allocation failed");
  }
  *out = c;
  return FDW_OK;
}

extern "C" int fdw_closure_destroy(fdw_closure *c) {
  if (!c) return FDW_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  closure_free_train(c);
  cudaFree(c->pf); cudaFree(c->pb); cudaFree(c->grad); cudaFree(c->m); cudaFree(c->v);
  cudaFree(c->partial); cudaFree(c->loss_partial);
  cudaFree(c->xpair);
  cudaFree(c->x); cudaFree(c->ia1); cudaFree(c->ia2); cudaFree(c->base); cudaFree(c->s_dev); cudaFree(c->s_partial);
  cudaFree(c->x16); cudaFree(c->tc_out); cudaFree(c->tcw); cudaFree(c->umw);
  delete c;
  return FDW_OK;
}

extern "C" int fdw_closure_set_variant(fdw_closure *c, int variant) {
  if (!c || variant < 0 || variant > 2) return report_error(FDW_ERR_INVALID_ARG, "variant must be 0, 1 or 2");
  c->variant = variant;
  return FDW_OK;
}

extern "C" int fdw_closure_set_params(fdw_closure *c, const float *p, int ptr_is_device) {
  if (!c || !p) return report_error(FDW_ERR_INVALID_ARG, "NULL closure or parameters");
  cudaError_t e = cudaMemcpyAsync(c->pf, p, kNumParams * sizeof(float),
                                  ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    to_bf16_kernel<<<(kNumParams + 255) / 256, 256, 0, c->stream>>>(c->pf, c->pb, kNumParams);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->m, 0, kNumParams * sizeof(float), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->v, 0, kNumParams * sizeof(float), c->stream);
  if (e == cudaSuccess && !ptr_is_device) e = cudaStreamSynchronize(c->stream);
  c->adam_t = 0;
  if (e != cudaSuccess) return report_error(FDW_ERR_CUDA, "fdw_closure_set_params: %s", cudaGetErrorString(e));
  return FDW_OK;
}

extern "C" int fdw_closure_get_params(fdw_closure *c, float *p, int ptr_is_device) {
  if (!c || !p) return report_error(FDW_ERR_INVALID_ARG, "NULL closure or output");
  cudaError_t e = cudaMemcpyAsync(p, c->pf, kNumParams * sizeof(float),
                                  ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && !ptr_is_device) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return report_error(FDW_ERR_CUDA, "fdw_closure_get_params: %s", cudaGetErrorString(e));
  return FDW_OK;
}

static int check_batch(int batch, int S) {
  if (batch < 1 || S < 7 || S > 512) return report_error(FDW_ERR_INVALID_ARG, "batch >= 1 and 7 <= S <= 512");
  return FDW_OK;
}

extern "C" int fdw_closure_forward(fdw_closure *c, const float *x, int batch, int S, float *out) {
  if (!c || !x || !out) return report_error(FDW_ERR_INVALID_ARG, "NULL argument");
  int rc = check_batch(batch, S);
  if (!rc) rc = closure_reserve_train(c, batch, S);
  if (rc) return rc;
  cudaError_t e = closure_pair_forward(c, x, batch, S);
  if (e == cudaSuccess) {
    const long long n3 = (long long)batch * (S - 6) * (S - 6) * (S - 6);
    pair_diff_kernel<<<grid_for(n3), 256, 0, c->stream>>>(c->out, n3, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return report_error(FDW_ERR_CUDA, "fdw_closure_forward: %s", cudaGetErrorString(e));
  return FDW_OK;
}

// loss (device float) and gradient (c->grad) of a batch
static int closure_loss_grad_impl(fdw_closure *c, const float *x, const float *t, int batch, int S,
                                  float *loss, bool want_grad) {
  int rc = check_batch(batch, S);
  if (!rc) rc = closure_reserve_train(c, batch, S);
  if (rc) return rc;
  cudaError_t e = closure_pair_forward(c, x, batch, S);
  const long long n3 = (long long)batch * (S - 6) * (S - 6) * (S - 6);
  const int nb = 1024;
  if (e == cudaSuccess) {
    mse_pair_kernel<<<nb, 256, 0, c->stream>>>(c->out, t, n3, (float)(1.0 / (double)n3), c->g3, c->loss_partial);
    sum_partials_kernel<<<1, 32, 0, c->stream>>>(c->loss_partial, nb, loss);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && want_grad)
    e = closure_backward_batch(c->xpair, c->pb, 2 * batch, S, c->a1, c->a2, c->g3, c->g2, c->g1, c->partial,
                               c->grad, c->stream);
  if (e != cudaSuccess) return report_error(FDW_ERR_CUDA, "closure loss/gradient: %s", cudaGetErrorString(e));
  return FDW_OK;
}

extern "C" int fdw_closure_loss_grad(fdw_closure *c, const float *x, const float *target, int batch, int S,
                                     float *loss, float *grad) {
  if (!c || !x || !target || !loss) return report_error(FDW_ERR_INVALID_ARG, "NULL argument");
  int rc = closure_loss_grad_impl(c, x, target, batch, S, loss, grad != nullptr);
  if (rc || !grad) return rc;
  if (cudaMemcpyAsync(grad, c->grad, kNumParams * sizeof(float), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
    return report_error(FDW_ERR_CUDA, "fdw_closure_loss_grad: copy");
  return FDW_OK;
}

extern "C" int fdw_closure_adam_step(fdw_closure *c, const float *x, const float *target, int batch, int S,
                                     float lr, float *loss) {
  if (!c || !x || !target || !loss || !(lr > 0.f)) return report_error(FDW_ERR_INVALID_ARG, "bad argument");
  int rc = closure_loss_grad_impl(c, x, target, batch, S, loss, true);
  if (rc) return rc;
  c->adam_t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const double c1 = 1.0 - pow(b1, (double)c->adam_t), c2 = 1.0 - pow(b2, (double)c->adam_t);
  adam_kernel<<<(kNumParams + 255) / 256, 256, 0, c->stream>>>(
      c->pf, c->grad, c->m, c->v, c->pb, kNumParams, lr, (float)b1, (float)(1.0 - b1), (float)b2,
      (float)(1.0 - b2), 1e-8f, (float)c1, (float)c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report_error(FDW_ERR_CUDA, "fdw_closure_adam_step: %s", cudaGetErrorString(e));
  return FDW_OK;
}
