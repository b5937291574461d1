// tti.cu -- the TTI pseudo-acoustic time step (Eq. TTI with the rotated
// operators of Eq. DiffOp and the fused sponge) for sm_103a.
//
//   P p+ = 2p - Q p- + c [ e H p + d G r ]
//   P r+ = 2r - Q r- + c [ d H p + G r ]
//   G = Gzz = sum_ij n_i n_j D_ij,  H = Gxx + Gyy = lap - Gzz,
//   e = 1 + 2 eps, d = sqrt(1 + 2 delta), n = (sin t cos f, sin t sin f, cos t).
// D_ii is the k-point second-derivative stencil, D_ij (i != j) the tensor
// product of the k-point first-derivative stencils. Gxx + Gyy + Gzz equals
// the Laplacian exactly (the rotated axes are orthonormal), so H is formed
// as lap - G without the other two rotated operators.
#include "fdw_internal.h"
#include "fdwave.h"
#include "ptx.cuh"

#include <string.h>

namespace fdw {

// One thread per point, plain global loads: the cross derivatives are the
// full (2r)^2-tap tensor products. A GPU cross-check of the 2.5D kernel of
// tti_kernel.cuh (instantiated per storage in tti_{f32,bf16,f16}.cu).
template <typename T, int R>
__global__ void __launch_bounds__(256)
    tti_naive_kernel(const T *__restrict__ pc, T *__restrict__ pp, const T *__restrict__ rc,
                     T *__restrict__ rp, const T *__restrict__ c, const T *__restrict__ e,
                     const T *__restrict__ dl, const T *__restrict__ ax,
                     const T *__restrict__ ay, Dims d, Weights w, Sponge sp) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= d.NX || y >= d.NY || z >= d.NZ) return;
  const size_t plane = d.plane();
  auto at = [&](const T *f, int xx, int yy, int zz) -> float {
    if (xx < 0 || yy < 0 || zz < 0 || xx >= d.NX || yy >= d.NY || zz >= d.NZ) return 0.f;
    return St<T>::ld(f[(size_t)zz * plane + (size_t)yy * d.Xp + xx]);
  };
  const size_t p = (size_t)z * plane + (size_t)y * d.Xp + x;
  const float nx_ = St<T>::ld(ax[p]), ny_ = St<T>::ld(ay[p]);
  const float nz_ = sqrtf(fmaxf(0.f, 1.f - nx_ * nx_ - ny_ * ny_));
  float lap[2], G[2];
  const T *fs[2] = {pc, rc};
#pragma unroll 1
  for (int f = 0; f < 2; ++f) {
    const T *u = fs[f];
    const float uc = at(u, x, y, z);
    float dxx = w.w2[0] * uc, dyy = w.w2[0] * uc, dzz = w.w2[0] * uc;
    float dxy = 0.f, dxz = 0.f, dyz = 0.f;
#pragma unroll 1
    for (int m = 1; m <= R; ++m) {
      dxx = fmaf(w.w2[m], at(u, x + m, y, z) + at(u, x - m, y, z), dxx);
      dyy = fmaf(w.w2[m], at(u, x, y + m, z) + at(u, x, y - m, z), dyy);
      dzz = fmaf(w.w2[m], at(u, x, y, z + m) + at(u, x, y, z - m), dzz);
#pragma unroll 1
      for (int n = 1; n <= R; ++n) {
        const float cc = w.c1[m] * w.c1[n];
        dxy = fmaf(cc, at(u, x + m, y + n, z) - at(u, x + m, y - n, z) - at(u, x - m, y + n, z) +
                           at(u, x - m, y - n, z), dxy);
        dxz = fmaf(cc, at(u, x + m, y, z + n) - at(u, x + m, y, z - n) - at(u, x - m, y, z + n) +
                           at(u, x - m, y, z - n), dxz);
        dyz = fmaf(cc, at(u, x, y + m, z + n) - at(u, x, y + m, z - n) - at(u, x, y - m, z + n) +
                           at(u, x, y - m, z - n), dyz);
      }
    }
    lap[f] = dxx + dyy + dzz;
    G[f] = nx_ * nx_ * dxx + ny_ * ny_ * dyy + nz_ * nz_ * dzz +
           2.f * (nx_ * ny_ * dxy + nx_ * nz_ * dxz + ny_ * nz_ * dyz);
  }
  const float Hp = lap[0] - G[0];
  const float gh = sp.gx[x] + sp.gy[y] + sp.gz[z];
  const float inv = __frcp_rn(1.f + gh), q = 1.f - gh;
  const float cc = St<T>::ld(c[p]), ee = St<T>::ld(e[p]), dd = St<T>::ld(dl[p]);
  const float p_new = (2.f * at(pc, x, y, z) - q * St<T>::ld(pp[p]) + cc * (ee * Hp + dd * G[1])) * inv;
  const float r_new = (2.f * at(rc, x, y, z) - q * St<T>::ld(rp[p]) + cc * (dd * Hp + G[1])) * inv;
  pp[p] = St<T>::st(p_new);
  rp[p] = St<T>::st(r_new);
}

template <typename T, int R>
static cudaError_t launch_r(const TTILaunch &L, cudaStream_t st) {
  dim3 blk(32, 8), grd((L.d.NX + 31) / 32, (L.d.NY + 7) / 8, L.d.NZ);
  tti_naive_kernel<T, R><<<grd, blk, 0, st>>>(
      (const T *)L.p_cur, (T *)L.p_prev, (const T *)L.r_cur, (T *)L.r_prev, (const T *)L.c,
      (const T *)L.e, (const T *)L.dl, (const T *)L.ax, (const T *)L.ay, L.d, L.w, L.sp);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_naive_t(const TTILaunch &L, cudaStream_t st) {
  switch (L.r) {
    case 1: return launch_r<T, 1>(L, st);
    case 2: return launch_r<T, 2>(L, st);
    case 3: return launch_r<T, 3>(L, st);
    case 4: return launch_r<T, 4>(L, st);
    case 5: return launch_r<T, 5>(L, st);
    case 6: return launch_r<T, 6>(L, st);
    case 7: return launch_r<T, 7>(L, st);
    case 8: return launch_r<T, 8>(L, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tti(const TTILaunch &L, cudaStream_t st) {
  if (L.naive && !L.prepare_only) {
    switch (L.storage) {
      case FDW_F32: return launch_naive_t<float>(L, st);
      case FDW_BF16: return launch_naive_t<__nv_bfloat16>(L, st);
      case FDW_F16: return launch_naive_t<__half>(L, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (L.storage) {
    case FDW_F32: return launch_tti_tma_f32(L, st);
    case FDW_BF16: return launch_tti_tma_bf16(L, st);
    case FDW_F16: return launch_tti_tma_f16(L, st);
    default: return cudaErrorInvalidValue;
  }
}

int tti_geom(int storage, int r, int tile, TileGeom *g) {
  switch (storage) {
    case FDW_F32: return tti_geom_f32(r, tile, g);
    case FDW_BF16: return tti_geom_bf16(r, tile, g);
    case FDW_F16: return tti_geom_f16(r, tile, g);
    default: return -1;
  }
}

// Default configuration (measured on the 464^3 TTI workload): four warps
// per CTA (they beat 2 and 8); up to order 8 the field-pair kernel: at
// order 6 two rows per thread with z unrolling 2, otherwise one row with z
// unrolling 4 for FP32 and two rows with z unrolling 1 for 16-bit storage
// (whose conversions make the shared y taps pay); above order 8 the scalar
// kernel with z unrolling 2 at orders 10-12 and 1 higher (the queues of 6
// fields grow with the order and the pairs' extra registers cost occupancy).
int tti_default_tile(int storage, int r) {
  if (r == 3) return 9;
  if (r <= 4) return storage == FDW_F32 ? 7 : 10;
  return r <= 6 ? 2 : 4;
}

int tti_ctas_per_sm(int storage, int r, int tile) {
  int occ = 0;
  TTILaunch L{};
  memset(&L, 0, sizeof L);
  L.storage = storage;
  L.r = r;
  L.tile = tile;
  L.prepare_only = 1;
  L.occupancy_out = &occ;
  if (launch_tti(L, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

cudaError_t tti_prepare(int storage, int r, int tile) {
  TTILaunch L{};
  memset(&L, 0, sizeof L);
  L.storage = storage;
  L.r = r;
  L.tile = tile;
  L.prepare_only = 1;
  return launch_tti(L, 0);
}

}  // namespace fdw
