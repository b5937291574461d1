// acoustic.cu -- dispatch of the acoustic time step (Algorithm 1 with
// Eq. Acou and the fused sponge): the 2.5D TMA kernel (acoustic_kernel.cuh,
// instantiated per storage type in acoustic_{f32,bf16,f16}.cu) and a
// one-thread-per-point kernel kept as an independent GPU cross-check.
#include <string.h>

#include "fdw_internal.h"
#include "fdwave.h"

namespace fdw {

// One thread per point, plain global loads with bounds checks.
template <typename T, int R>
__global__ void __launch_bounds__(256)
    acoustic_naive_kernel(const T *cur, const T *prev, T *out, const T *__restrict__ c, Dims d, Weights w,
                          Sponge sp) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= d.NX || y >= d.NY || z >= d.NZ) return;
  const size_t plane = d.plane();
  auto at = [&](int xx, int yy, int zz) -> float {
    if (xx < 0 || yy < 0 || zz < 0 || xx >= d.NX || yy >= d.NY || zz >= d.NZ) return 0.f;
    return St<T>::ld(cur[(size_t)zz * plane + (size_t)yy * d.Xp + xx]);
  };
  const float uc = at(x, y, z);
  float lx = 0.f, ly = 0.f, lz = 0.f;
#pragma unroll
  for (int m = 1; m <= R; ++m) {
    lx = fmaf(w.w2[m], at(x + m, y, z) + at(x - m, y, z), lx);
    ly = fmaf(w.w2[m], at(x, y + m, z) + at(x, y - m, z), ly);
    lz = fmaf(w.w2[m], at(x, y, z + m) + at(x, y, z - m), lz);
  }
  const float lap = fmaf(3.f * w.w2[0], uc, lx + ly + lz);
  const size_t p = (size_t)z * plane + (size_t)y * d.Xp + x;
  const float gh = sp.gx[x] + sp.gy[y] + sp.gz[z];
  const float up =
      (2.f * uc - (1.f - gh) * St<T>::ld(prev[p]) + St<T>::ld(c[p]) * lap) * __frcp_rn(1.f + gh);
  out[p] = St<T>::st(up);
}

template <typename T, int R>
static cudaError_t launch_naive_r(const AcousticLaunch &L, cudaStream_t st) {
  dim3 blk(32, 8), grd((L.d.NX + 31) / 32, (L.d.NY + 7) / 8, L.d.NZ);
  acoustic_naive_kernel<T, R><<<grd, blk, 0, st>>>((const T *)L.cur, (const T *)L.prev,
                                                   (T *)(L.out ? L.out : L.prev), (const T *)L.c, L.d, L.w,
                                                   L.sp);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_naive(const AcousticLaunch &L, cudaStream_t st) {
  switch (L.r) {
    case 1: return launch_naive_r<T, 1>(L, st);
    case 2: return launch_naive_r<T, 2>(L, st);
    case 3: return launch_naive_r<T, 3>(L, st);
    case 4: return launch_naive_r<T, 4>(L, st);
    case 5: return launch_naive_r<T, 5>(L, st);
    case 6: return launch_naive_r<T, 6>(L, st);
    case 7: return launch_naive_r<T, 7>(L, st);
    case 8: return launch_naive_r<T, 8>(L, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_acoustic(const AcousticLaunch &L, cudaStream_t st) {
  if (L.naive && !L.prepare_only) {
    switch (L.storage) {
      case FDW_F32: return launch_naive<float>(L, st);
      case FDW_BF16: return launch_naive<__nv_bfloat16>(L, st);
      case FDW_F16: return launch_naive<__half>(L, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (L.storage) {
    case FDW_F32: return launch_acoustic_f32(L, st);
    case FDW_BF16: return launch_acoustic_bf16(L, st);
    case FDW_F16: return launch_acoustic_f16(L, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t acoustic_prepare(int storage, int r, int tile) {
  AcousticLaunch L{};
  L.storage = storage;
  L.r = r;
  L.tile = tile;
  L.prepare_only = 1;
  return launch_acoustic(L, 0);
}

int acoustic_ctas_per_sm(int storage, int r, int tile) {
  int occ = 0;
  AcousticLaunch L{};
  L.storage = storage;
  L.r = r;
  L.tile = tile;
  L.prepare_only = 1;
  L.occupancy_out = &occ;
  if (launch_acoustic(L, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

int acoustic_geom(int storage, int r, int tile, TileGeom *g) {
  switch (storage) {
    case FDW_F32: return acoustic_geom_f32(r, tile, g);
    case FDW_BF16: return acoustic_geom_bf16(r, tile, g);
    case FDW_F16: return acoustic_geom_f16(r, tile, g);
    default: return -1;
  }
}

// Default configuration per (storage, radius): the fastest on the 592^3
// workload in sweeps of the configurations (default z chunking) at every
// even order 2-16 for FP32 and at orders 2, 4, 8, 12, 16 for 16-bit
// storage (radii 3, 5 and 7 take a neighbour's choice there).
int acoustic_default_tile(int storage, int r) {
  static const int best32[kMaxR + 1] = {1, 1, 3, 3, 10, 10, 10, 10, 6};
  static const int best16[kMaxR + 1] = {1, 1, 1, 1, 1, 5, 5, 5, 5};
  if (r < 1 || r > kMaxR) return 1;
  return storage == FDW_F32 ? best32[r] : best16[r];
}

}  // namespace fdw
