// acoustic_kernel.cuh -- the 2.5D z-marching acoustic step kernel (template).
//
//   P u+ = 2u - Q u- + c lap_h(u),   c = (v dt / h)^2, P,Q = 1 +- gamma dt/2
//   lap_h(u) = sum over x, y, z of [w0 u + sum_{m=1..r} w_m (u_{+m} + u_{-m})]
//
// The star stencil of width k = 2r+1 per axis (Section "Stencil operators");
// the paper counts 16 B of DRAM traffic per point for it (read u_n, u_{n-1},
// the medium; write u_{n+1}: Table 1 / Eq. eqn_oi with l + s = 4 fields).
//
// Geometry. A CTA owns a TX x TY column of the grid (TX = 32 RX, TY = BY RY)
// and marches a chunk of z planes. Thread (tx, ty) owns RX consecutive x
// points in each of RY consecutive rows. Per plane:
//   * x neighbours: the thread loads its row segment [RX tx - RR, RX tx + RX
//     + RR) from the shared-memory halo tile as RX-wide vectors and folds
//     each element into the RX point sums as it arrives (RR = r rounded up
//     to RX);
//   * y neighbours: rows ty RY - r .. ty RY + RY - 1 + r are loaded once as
//     RX-wide vectors and folded into the RY x RX point sums;
//   * z neighbours: a register queue of 2r + U planes per point; the z loop
//     is unrolled U times so the queue shifts by U planes (2r moves) every U
//     planes instead of every plane.
// With RX even the point sums run on packed FP32 pairs (Pk<2> below).
// TMA keeps NS stages in flight, each an mbarrier-tracked slot holding the
// interior tile of plane z+r (queue head), and the halo tile, u_{n-1} tile
// and c tile of output plane z. u_{n+1} goes straight from registers to
// HBM with RX-wide coalesced stores. Damping comes from three 1D tables.
// Every mbarrier wait is bounded: a CTA that gives up sets the error flag,
// drains its own copies (bounded) and exits.
#pragma once

#include "fdw_internal.h"
#include "fdwave.h"
#include "ptx.cuh"

namespace fdw {

template <typename T, int N> struct alignas(sizeof(T) * N) Vec {
  T v[N];
};

// Packed FP32 arithmetic. With an even number of x points per thread the
// kernel handles them in pairs through the f32x2 instructions (__ffma2_rn,
// __fadd2_rn, __fmul2_rn: per component the rounding of the scalar
// operation), halving the issue slots of the stencil arithmetic, which is
// what bounds the high orders. Pk<1> is the scalar fallback (RX = 1).
template <int W> struct Pk;
template <> struct Pk<1> {
  using E = float;
  static __device__ __forceinline__ E fma(E a, E b, E c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ E add(E a, E b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ E mul(E a, E b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ E splat(float a) { return a; }
  static __device__ __forceinline__ E make(float a, float) { return a; }
  static __device__ __forceinline__ float &at(E &e, int) { return e; }
  static __device__ __forceinline__ float get(const E &e, int) { return e; }
  static __device__ __forceinline__ E wt(const Weights &w, int m) { return w.w2[m]; }
};
template <> struct Pk<2> {
  using E = float2;
  static __device__ __forceinline__ E fma(E a, E b, E c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ E add(E a, E b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ E mul(E a, E b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ E splat(float a) { return make_float2(a, a); }
  static __device__ __forceinline__ E make(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ float &at(E &e, int i) { return i ? e.y : e.x; }
  static __device__ __forceinline__ float get(const E &e, int i) { return i ? e.y : e.x; }
  static __device__ __forceinline__ E wt(const Weights &w, int m) { return w.w2p[m]; }
};

template <typename T, int R, int RX, int RY, int BY, int NS, int U, int BP = 1>
struct AcTile {
  static constexpr int TX = 32 * RX;
  static constexpr int TY = BY * RY;
  static constexpr int EL = (int)sizeof(T);
  static constexpr int XALIGN = 16 / EL;  // TMA: x * element size multiple of 16 B
  static constexpr int RR = ((R + RX - 1) / RX) * RX;
  static constexpr int HX = ((RR + XALIGN - 1) / XALIGN) * XALIGN;
  static constexpr int BXH = TX + 2 * HX;
  static constexpr int BYH = TY + 2 * R;
  static constexpr int a128(int b) { return (b + 127) / 128 * 128; }
  static constexpr int HALO_B = a128(BXH * BYH * EL);
  static constexpr int INT_B = a128(TX * TY * EL);
  static constexpr int STAGE_B = HALO_B + 3 * INT_B;  // halo | head | prev | c
  static constexpr int BAR_B = 128;
  static constexpr int SMEM_B = NS * STAGE_B + BAR_B + kMaxZChunk * 4 + 128;
  static constexpr int THREADS = 32 * BY;
  static constexpr int QL = 2 * R + U;
  static_assert(NS >= 2, "ring needs two stages");
  static_assert(BP >= 1 && U % BP == 0 && NS > BP, "barrier period divides the unroll, ring deeper than it");
  static_assert(BXH <= 256 && BYH <= 256 && TX <= 256 && TY <= 256, "TMA box dimension limit");
  static_assert((BXH * EL) % 16 == 0 && (TX * EL) % 16 == 0, "TMA inner box bytes");
  static_assert((HX * EL) % 16 == 0, "TMA x coordinate alignment");
  static_assert(HX % RX == 0 && HX >= RR, "vector loads stay inside the halo tile");
  static_assert(SMEM_B <= 227 * 1024, "shared memory per CTA");
};

template <typename T, int R, int RX, int RY, int BY, int NS, int U, int BP>
__global__ void __launch_bounds__(32 * BY)
    acoustic_tma_kernel(const __grid_constant__ CUtensorMap m_halo,
                        const __grid_constant__ CUtensorMap m_head,
                        const __grid_constant__ CUtensorMap m_prev,
                        const __grid_constant__ CUtensorMap m_c, T *__restrict__ out, Dims d,
                        Weights w, Sponge sp, int zc, int *err) {
  using C = AcTile<T, R, RX, RY, BY, NS, U, BP>;
  using V = Vec<T, RX>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  uint64_t *bars = (uint64_t *)(smem + NS * C::STAGE_B);
  float *gzs = (float *)(smem + NS * C::STAGE_B + C::BAR_B);  // damping of this z chunk

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, d.NZ);
  if (z0 >= z1 || zc > kMaxZChunk) return;  // uniform over the CTA (the host bounds zc)
  const int nit = (z1 - z0) + 2 * R;
  const int xl = RX * tx;  // first x of this thread inside the tile
  // x / y damping of the thread's points, constant over the march
  float gxr[RX], gyr[RY];
#pragma unroll
  for (int rx = 0; rx < RX; ++rx) gxr[rx] = (x0 + xl + rx < d.NX) ? sp.gx[x0 + xl + rx] : 0.f;
#pragma unroll
  for (int ry = 0; ry < RY; ++ry) gyr[ry] = (y0 + ty * RY + ry < d.NY) ? sp.gy[y0 + ty * RY + ry] : 0.f;

  if (tid == 0) {
    prefetch_tensormap(&m_halo);
    prefetch_tensormap(&m_head);
    prefetch_tensormap(&m_prev);
    prefetch_tensormap(&m_c);
#pragma unroll
    for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
    fence_barrier_init();
  }
  for (int i = tid; i < z1 - z0; i += C::THREADS) gzs[i] = sp.gz[z0 + i];
  __syncthreads();

  // Stage j: head plane zh = z0 - R + j (if inside the grid) and, once the
  // queue is full (j >= 2R), output plane zo = zh - R with halo/prev/c.
  int issued_hi = -1;  // meaningful in thread 0 only
  auto issue = [&](int j) {
    const int s = j % NS;
    const int zh = z0 - R + j;
    const bool head = (zh >= 0 && zh < d.NZ);
    const bool outp = (j >= 2 * R);
    const uint32_t bytes = (head ? C::TX * C::TY * C::EL : 0) +
                           (outp ? (C::BXH * C::BYH + 2 * C::TX * C::TY) * C::EL : 0);
    const uint32_t bar = smem_u32(&bars[s]);
    unsigned char *st = smem + s * C::STAGE_B;
    mbar_arrive_expect_tx(bar, bytes);
    if (head) tma_load_3d(smem_u32(st + C::HALO_B), &m_head, x0, y0, zh, bar);
    if (outp) {
      const int zo = zh - R;
      tma_load_3d(smem_u32(st), &m_halo, x0 - C::HX, y0 - R, zo, bar);
      tma_load_3d(smem_u32(st + C::HALO_B + C::INT_B), &m_prev, x0, y0, zo, bar);
      tma_load_3d(smem_u32(st + C::HALO_B + 2 * C::INT_B), &m_c, x0, y0, zo, bar);
    }
    issued_hi = j;
  };
  if (tid == 0) {
    const int n0 = nit < NS ? nit : NS;
    for (int j = 0; j < n0; ++j) issue(j);
  }

  // Points are handled in packs of W (pairs when RX is even): pack k holds
  // x points W k .. W k + W - 1 of the thread's row segment.
  constexpr int W = (RX % 2 == 0) ? 2 : 1;
  constexpr int NK = RX / W;
  using P = Pk<W>;
  using E = typename P::E;
  // q[ry][k][s]: slots u..u+2R hold planes zh+u-2R .. zh+u during
  // sub-iteration u of a group of U planes.
  E q[RY][NK][C::QL];
#pragma unroll
  for (int ry = 0; ry < RY; ++ry)
#pragma unroll
    for (int k = 0; k < NK; ++k)
#pragma unroll
      for (int i = 0; i < C::QL; ++i) q[ry][k][i] = P::splat(0.f);

  const E wc = P::splat(3.f * w.w2[0]);
  const size_t plane = d.plane();
  // a bounded wait that gave up between barriers (BP > 1)
  bool bad = false;
  int bad_at = 0;

#pragma unroll 1
  for (int j0 = 0; j0 < nit; j0 += U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u;
      if (j >= nit) break;  // uniform
      const int s = j % NS;
      const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((j / NS) & 1));
      if (u % BP == 0) {
        // The CTA barrier, every BP planes: every thread has finished the
        // iterations before j, so their BP stages can be refilled.
        if (__syncthreads_or(bad || !ok)) {
          if (tid == 0) {
            atomicOr(err, kErrWaitTimeout);
            for (int jj = bad_at; jj <= issued_hi; ++jj)
              (void)mbar_wait_bounded(smem_u32(&bars[jj % NS]), (uint32_t)((jj / NS) & 1));
          }
          return;
        }
        if (tid == 0) {
#pragma unroll
          for (int k = BP; k >= 1; --k)
            if (j - k >= 0 && j - k + NS < nit) issue(j - k + NS);
        }
      } else if (!ok && !bad) {
        // the CTA leaves at the next barrier; until then this thread's
        // results are not valid (the error flag says so) but every access
        // stays inside the tile and the output field
        bad = true;
        bad_at = j;
      }

      const unsigned char *st = smem + s * C::STAGE_B;
      const int zh = z0 - R + j;
      const bool head = (zh >= 0 && zh < d.NZ);
      const T *hd = (const T *)(st + C::HALO_B);
#pragma unroll
      for (int ry = 0; ry < RY; ++ry) {
        V v;
        if (head) v = *(const V *)(hd + (ty * RY + ry) * C::TX + xl);
#pragma unroll
        for (int k = 0; k < NK; ++k)
          q[ry][k][2 * R + u] =
              head ? P::make(St<T>::ld(v.v[W * k]), St<T>::ld(v.v[W * k + W - 1])) : P::splat(0.f);
      }
      if (j < 2 * R) continue;

      const int zo = zh - R;
      const T *H = (const T *)st;
      const T *PV = (const T *)(st + C::HALO_B + C::INT_B);
      const T *CC = (const T *)(st + C::HALO_B + 2 * C::INT_B);

      E acc[RY][NK];
      // z direction and centre, from the queue
#pragma unroll
      for (int ry = 0; ry < RY; ++ry)
#pragma unroll
        for (int k = 0; k < NK; ++k) {
          E a = P::mul(wc, q[ry][k][u + R]);
#pragma unroll
          for (int m = 1; m <= R; ++m)
            a = P::fma(P::wt(w, m), P::add(q[ry][k][u + R + m], q[ry][k][u + R - m]), a);
          acc[ry][k] = a;
        }
      // y direction: rows ty RY - R .. ty RY + RY - 1 + R of the halo tile
#pragma unroll
      for (int t = -R; t < RY + R; ++t) {
        const V v = *(const V *)(H + (ty * RY + t + R) * C::BXH + C::HX + xl);
#pragma unroll
        for (int ry = 0; ry < RY; ++ry) {
          const int m = t - ry < 0 ? ry - t : t - ry;
          if (m >= 1 && m <= R) {
#pragma unroll
            for (int k = 0; k < NK; ++k)
              acc[ry][k] = P::fma(P::wt(w, m), P::make(St<T>::ld(v.v[W * k]), St<T>::ld(v.v[W * k + W - 1])),
                                  acc[ry][k]);
          }
        }
      }
      // x direction: the row segment of each of the thread's rows. Taps at
      // an even distance pair up aligned elements (x_e, x_e+1) with the
      // points (W k, W k + 1); odd distances go component by component.
#pragma unroll
      for (int ry = 0; ry < RY; ++ry) {
        const T *row = H + (ty * RY + ry + R) * C::BXH + C::HX + xl;
#pragma unroll
        for (int o = -C::RR; o < RX + C::RR; o += RX) {
          const V v = *(const V *)(row + o);
#pragma unroll
          for (int e = 0; e < RX; e += W) {
#pragma unroll
            for (int k = 0; k < NK; ++k) {
              const int t = o + e - W * k;
              const int m = t < 0 ? -t : t;
              if (m >= 1 && m <= R)
                acc[ry][k] = P::fma(P::wt(w, m), P::make(St<T>::ld(v.v[e]), St<T>::ld(v.v[e + W - 1])),
                                    acc[ry][k]);
            }
          }
          if constexpr (W == 2) {
#pragma unroll
            for (int e = 0; e < RX; ++e) {
#pragma unroll
              for (int k = 0; k < NK; ++k) {
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                  const int t = o + e - 2 * k - i;
                  const int m = t < 0 ? -t : t;
                  if ((m & 1) && m <= R)
                    P::at(acc[ry][k], i) = fmaf(w.w2[m], St<T>::ld(v.v[e]), P::at(acc[ry][k], i));
                }
              }
            }
          }
        }
      }
      // update and store: u+ = (2u - (1 - g) u- + c lap u) / (1 + g) with
      // g = gamma dt / 2; 1/(1 + g) by the fast reciprocal (<= 2 ulp;
      // exactly 1 outside the sponge). Pairs of points on f32x2.
      const float ghz = gzs[zo - z0];
#pragma unroll
      for (int ry = 0; ry < RY; ++ry) {
        const int yl = ty * RY + ry;
        const V vm = *(const V *)(PV + yl * C::TX + xl);
        const V vc = *(const V *)(CC + yl * C::TX + xl);
        const float gyz = gyr[ry] + ghz;
        V res;
#pragma unroll
        for (int k = 0; k < NK; ++k) {
          const E gh = P::add(P::make(gxr[W * k], gxr[W * k + W - 1]), P::splat(gyz));
          const E uc = q[ry][k][u + R];
          E t = P::fma(P::make(St<T>::ld(vc.v[W * k]), St<T>::ld(vc.v[W * k + W - 1])), acc[ry][k],
                       P::add(uc, uc));
          t = P::fma(P::add(gh, P::splat(-1.f)), P::make(St<T>::ld(vm.v[W * k]), St<T>::ld(vm.v[W * k + W - 1])),
                     t);
          const E up = P::mul(t, P::make(__fdividef(1.f, 1.f + P::get(gh, 0)),
                                         __fdividef(1.f, 1.f + P::get(gh, W - 1))));
#pragma unroll
          for (int i = 0; i < W; ++i) res.v[W * k + i] = St<T>::st(P::get(up, i));
        }
        const int x = x0 + xl, y = y0 + yl;
        if (y < d.NY) {
          T *dst = out + (size_t)zo * plane + (size_t)y * d.Xp + x;
          if (x + RX <= d.NX) {
            *(V *)dst = res;
          } else {
#pragma unroll
            for (int rx = 0; rx < RX; ++rx)
              if (x + rx < d.NX) dst[rx] = res.v[rx];
          }
        }
      }
    }
    // shift the queue by U planes
#pragma unroll
    for (int ry = 0; ry < RY; ++ry)
#pragma unroll
      for (int k = 0; k < NK; ++k)
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) q[ry][k][i] = q[ry][k][i + U];
  }
  if (bad) {  // gave up after the last barrier
    atomicOr(err, kErrWaitTimeout);
    if (tid == 0)
      for (int jj = bad_at; jj <= issued_hi; ++jj)
        (void)mbar_wait_bounded(smem_u32(&bars[jj % NS]), (uint32_t)((jj / NS) & 1));
  }
}

// Host-side launch of one configuration.
template <typename T, int R, int RX, int RY, int BY, int NS, int U, int BP>
cudaError_t launch_acoustic_cfg(const AcousticLaunch &L, cudaStream_t st) {
  using C = AcTile<T, R, RX, RY, BY, NS, U, BP>;
  auto kern = acoustic_tma_kernel<T, R, RX, RY, BY, NS, U, BP>;
  if (L.prepare_only) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_B);
    if (e == cudaSuccess && L.occupancy_out)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(L.occupancy_out, kern, C::THREADS, C::SMEM_B);
    return e;
  }
  const int zch = L.zchunks < 1 ? 1 : L.zchunks;
  const int zc = (L.d.NZ + zch - 1) / zch;
  if (zc > kMaxZChunk) return cudaErrorInvalidValue;
  dim3 grd((L.d.NX + C::TX - 1) / C::TX, (L.d.NY + C::TY - 1) / C::TY, (L.d.NZ + zc - 1) / zc);
  dim3 blk(32, BY);
  kern<<<grd, blk, C::SMEM_B, st>>>(*L.map_cur_halo, *L.map_cur_int, *L.map_prev_int, *L.map_c_int,
                                     (T *)(L.out ? L.out : L.prev), L.d, L.w, L.sp, zc, L.err);
  return cudaGetLastError();
}

template <typename T, int R, int RX, int RY, int BY, int NS, int U, int BP>
void tile_cfg(TileGeom *g) {
  using C = AcTile<T, R, RX, RY, BY, NS, U, BP>;
  g->box_halo_x = C::BXH;
  g->box_halo_y = C::BYH;
  g->box_int_x = C::TX;
  g->box_int_y = C::TY;
  g->smem = C::SMEM_B;
}

// Candidate configurations (RX, RY, BY, U, BP, NS), selected at run time by
// index; BP = planes per CTA barrier, NS = TMA ring stages (3 stages leave
// room for a third CTA per SM where the registers allow it).
#define FDW_AC_CFGS(X)    \
  X(0, 1, 4, 4, 1, 1, 4)  \
  X(1, 4, 2, 4, 4, 1, 4)  \
  X(2, 4, 1, 8, 4, 1, 4)  \
  X(3, 2, 2, 8, 4, 1, 4)  \
  X(4, 4, 2, 8, 2, 1, 4)  \
  X(5, 4, 2, 4, 2, 1, 4)  \
  X(6, 4, 2, 4, 4, 2, 4)  \
  X(7, 2, 2, 8, 4, 2, 4)  \
  X(8, 4, 1, 8, 4, 2, 4)  \
  X(9, 4, 2, 4, 4, 2, 3)  \
  X(10, 4, 2, 4, 4, 1, 3) \
  X(11, 2, 2, 8, 4, 2, 3) \
  X(12, 4, 2, 4, 2, 2, 4)

// Per-storage dispatch over radius and configuration (one TU per storage).
#define FDW_AC_DEFINE_STORAGE(SUFFIX, TYPE)                                                   \
  template <int R>                                                                            \
  static cudaError_t launch_r_##SUFFIX(const AcousticLaunch &L, cudaStream_t st) {           \
    switch (L.tile) {                                                                         \
      FDW_AC_CFGS(FDW_AC_CASE_LAUNCH)                                                         \
      default: return cudaErrorInvalidValue;                                                  \
    }                                                                                         \
  }                                                                                           \
  template <int R>                                                                            \
  static int geom_r_##SUFFIX(int tile, TileGeom *g) {                                        \
    switch (tile) {                                                                           \
      FDW_AC_CFGS(FDW_AC_CASE_GEOM)                                                           \
      default: return -1;                                                                     \
    }                                                                                         \
  }                                                                                           \
  cudaError_t launch_acoustic_##SUFFIX(const AcousticLaunch &L, cudaStream_t st) {           \
    switch (L.r) {                                                                            \
      case 1: return launch_r_##SUFFIX<1>(L, st);                                             \
      case 2: return launch_r_##SUFFIX<2>(L, st);                                             \
      case 3: return launch_r_##SUFFIX<3>(L, st);                                             \
      case 4: return launch_r_##SUFFIX<4>(L, st);                                             \
      case 5: return launch_r_##SUFFIX<5>(L, st);                                             \
      case 6: return launch_r_##SUFFIX<6>(L, st);                                             \
      case 7: return launch_r_##SUFFIX<7>(L, st);                                             \
      case 8: return launch_r_##SUFFIX<8>(L, st);                                             \
      default: return cudaErrorInvalidValue;                                                  \
    }                                                                                         \
  }                                                                                           \
  int acoustic_geom_##SUFFIX(int r, int tile, TileGeom *g) {                                 \
    switch (r) {                                                                              \
      case 1: return geom_r_##SUFFIX<1>(tile, g);                                             \
      case 2: return geom_r_##SUFFIX<2>(tile, g);                                             \
      case 3: return geom_r_##SUFFIX<3>(tile, g);                                             \
      case 4: return geom_r_##SUFFIX<4>(tile, g);                                             \
      case 5: return geom_r_##SUFFIX<5>(tile, g);                                             \
      case 6: return geom_r_##SUFFIX<6>(tile, g);                                             \
      case 7: return geom_r_##SUFFIX<7>(tile, g);                                             \
      case 8: return geom_r_##SUFFIX<8>(tile, g);                                             \
      default: return -1;                                                                     \
    }                                                                                         \
  }

}  // namespace fdw

// Case bodies used by FDW_AC_DEFINE_STORAGE; StorageT is defined by the
// including translation unit.
#define FDW_AC_CASE_LAUNCH(ID, RX, RY, BY, U, BP, NS) \
  case ID: return launch_acoustic_cfg<StorageT, R, RX, RY, BY, NS, U, BP>(L, st);
#define FDW_AC_CASE_GEOM(ID, RX, RY, BY, U, BP, NS) \
  case ID: tile_cfg<StorageT, R, RX, RY, BY, NS, U, BP>(g); return 0;
