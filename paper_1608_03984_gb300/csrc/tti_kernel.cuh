// tti_kernel.cuh -- the 2.5D z-marching TTI step kernel (template).
//
// Eq. TTI with the rotated operators of Eq. DiffOp and the fused sponge:
//   P p+ = 2p - Q p- + c [ e H p + d G r ]
//   P r+ = 2r - Q r- + c [ d H p + G r ]
//   G f = sum_ij n_i n_j D_ij f,   H f = (Gxx + Gyy) f = lap f - G f,
// n = (sin t cos f, sin t sin f, cos t), e = 1 + 2 eps, d = sqrt(1 + 2 delta).
// D_ii is the k-point second-derivative stencil, D_ij (i != j) the tensor
// product of the k-point first-derivative stencils D_i D_j, evaluated here
// in factored form (first derivative of a first derivative): the same
// discrete operator with O(k) instead of O(k^2) operations per point.
//
// Geometry. A CTA owns a 32 x TY column (one point per thread; the field-pair
// kernel can also take RY = 2 consecutive rows per thread) and marches a
// chunk of z planes. Everything that needs x/y neighbours is computed when a
// plane enters the march as the HEAD plane z+r, from one TMA halo tile per
// field:
//   f_xx, f_yy, D_x f, D_y f, and D_x(D_y f) (through a shared scratch of
//   D_y f that includes the x halo), folded with that plane's axis into
//   A f = nx^2 f_xx + ny^2 f_yy + 2 nx ny f_xy   (in-plane part of G f);
// f, D_x f, D_y f enter register queues of 2r + U planes and the in-plane
// sums (f_xx + f_yy - A f for p, A f for r) a delay queue of r + U planes.
// When the plane is the OUTPUT plane z, the z parts follow from the queues:
//   f_zz, D_z(D_x f), D_z(D_y f), and
//   H p = [p_xx + p_yy - A p] + (1 - nz^2) p_zz - 2 nx nz p_xz - 2 ny nz p_yz
//   G r = [A r] + nz^2 r_zz + 2 nx nz r_xz + 2 ny nz r_yz.
// The axis is stored as (nx, ny) with nz = sqrt(1 - nx^2 - ny^2) >= 0
// (n n^T does not depend on the sign of n).
//
// Each TMA stage holds: the p and r halo tiles and the (nx, ny) tiles of the
// head plane; the p-, r-, c, e, d, nx, ny tiles of the output plane. The
// D_y scratch is double-buffered and the cross term D_x(D_y f) of a head
// plane is finished one iteration later, so one CTA barrier per plane (the
// ring's) orders both the stage reuse and the scratch. The D_y of the x
// halo columns is spread evenly over the warps. Every mbarrier wait is
// bounded (error flag, drain, exit).
#pragma once

#include "fdw_internal.h"
#include "fdwave.h"
#include "ptx.cuh"

namespace fdw {

template <typename T, int R, int BY, int NS, int U, bool SH = false, int RY = 1>
struct TtiTile {
  static constexpr int TX = 32;
  static constexpr int TY = BY * RY;  // RY rows per thread (field-pair kernel)
  static constexpr int EL = (int)sizeof(T);
  static constexpr int XALIGN = 16 / EL;
  static constexpr int HX = ((R + XALIGN - 1) / XALIGN) * XALIGN;
  static constexpr int BXH = TX + 2 * HX;
  static constexpr int BYH = TY + 2 * R;
  static constexpr int a128(int b) { return (b + 127) / 128 * 128; }
  static constexpr int HALO_B = a128(BXH * BYH * EL);
  static constexpr int INT_B = a128(TX * TY * EL);
  // slot: halo p | halo r | head nx, ny | out pm, rm, c, e, d, nx, ny
  static constexpr int N_INT = 9;
  static constexpr int STAGE_B = 2 * HALO_B + N_INT * INT_B;
  static constexpr int SY = TX + 2 * R;  // row length of the D_y scratch
  static constexpr int SCR_B = SH ? 0 : a128(2 * 2 * TY * SY * 4);  // [buffer][field][TY][SY]
  static constexpr int NHALO = 2 * 2 * R * TY;               // D_y halo items per plane
  static constexpr int HPW = (NHALO + BY - 1) / BY;          // items per warp
  static constexpr int BAR_B = 128;
  static constexpr int SMEM_B = NS * STAGE_B + SCR_B + BAR_B + kMaxZChunk * 4 + 128;
  static constexpr int THREADS = 32 * BY;
  static constexpr int QL = 2 * R + U;
  static constexpr int DL = R + U;
  static_assert(NS >= 2, "ring needs two stages");
  static_assert(BXH <= 256 && BYH <= 256, "TMA box dimension limit");
  static_assert((BXH * EL) % 16 == 0 && (TX * EL) % 16 == 0 && (HX * EL) % 16 == 0, "TMA alignment");
  static_assert(SMEM_B <= 227 * 1024, "shared memory per CTA");
  static_assert(RY > 1 || HPW <= 32, "one D_y halo item per lane");
  static_assert(2 * R <= 32, "shuffle variant: the row's D_y halo columns fit one warp");
};

template <typename T, int R, int BY, int NS, int U, bool SH>
__global__ void __launch_bounds__(32 * BY)
    tti_tma_kernel(const __grid_constant__ CUtensorMap m_ph, const __grid_constant__ CUtensorMap m_rh,
                   const __grid_constant__ CUtensorMap m_pm, const __grid_constant__ CUtensorMap m_rm,
                   const __grid_constant__ CUtensorMap m_c, const __grid_constant__ CUtensorMap m_e,
                   const __grid_constant__ CUtensorMap m_d, const __grid_constant__ CUtensorMap m_ax,
                   const __grid_constant__ CUtensorMap m_ay, T *__restrict__ p_out,
                   T *__restrict__ r_out, Dims d, Weights w, Sponge sp, int zc, int *err) {
  using C = TtiTile<T, R, BY, NS, U, SH>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  float *scr = (float *)(smem + NS * C::STAGE_B);  // [2][2][TY][SY] D_y of p and r
  uint64_t *bars = (uint64_t *)(smem + NS * C::STAGE_B + C::SCR_B);
  float *gzs = (float *)(smem + NS * C::STAGE_B + C::SCR_B + C::BAR_B);

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, d.NZ);
  if (z0 >= z1 || zc > kMaxZChunk) return;  // uniform over the CTA
  const int nit = (z1 - z0) + 2 * R;
  const float gxr = (x0 + tx < d.NX) ? sp.gx[x0 + tx] : 0.f;
  const float gyr = (y0 + ty < d.NY) ? sp.gy[y0 + ty] : 0.f;

  const CUtensorMap *maps_int[C::N_INT] = {&m_ax, &m_ay, &m_pm, &m_rm, &m_c, &m_e, &m_d, &m_ax, &m_ay};
  if (tid == 0) {
    prefetch_tensormap(&m_ph);
    prefetch_tensormap(&m_rh);
#pragma unroll
    for (int i = 0; i < 7; ++i) prefetch_tensormap(maps_int[2 + i]);
#pragma unroll
    for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
    fence_barrier_init();
  }
  for (int i = tid; i < z1 - z0; i += C::THREADS) gzs[i] = sp.gz[z0 + i];
  __syncthreads();

  int issued_hi = -1;
  auto issue = [&](int j) {
    const int s = j % NS;
    const int zh = z0 - R + j;
    const bool head = (zh >= 0 && zh < d.NZ);
    const bool outp = (j >= 2 * R);
    const uint32_t bytes = (head ? (2 * C::BXH * C::BYH + 2 * C::TX * C::TY) * C::EL : 0) +
                           (outp ? 7 * C::TX * C::TY * C::EL : 0);
    const uint32_t bar = smem_u32(&bars[s]);
    unsigned char *st = smem + s * C::STAGE_B;
    mbar_arrive_expect_tx(bar, bytes);
    if (head) {
      tma_load_3d(smem_u32(st), &m_ph, x0 - C::HX, y0 - R, zh, bar);
      tma_load_3d(smem_u32(st + C::HALO_B), &m_rh, x0 - C::HX, y0 - R, zh, bar);
      tma_load_3d(smem_u32(st + 2 * C::HALO_B + 0 * C::INT_B), &m_ax, x0, y0, zh, bar);
      tma_load_3d(smem_u32(st + 2 * C::HALO_B + 1 * C::INT_B), &m_ay, x0, y0, zh, bar);
    }
    if (outp) {
      const int zo = zh - R;
#pragma unroll
      for (int i = 2; i < C::N_INT; ++i)
        tma_load_3d(smem_u32(st + 2 * C::HALO_B + i * C::INT_B), maps_int[i], x0, y0, zo, bar);
    }
    issued_hi = j;
  };
  if (tid == 0) {
    const int n0 = nit < NS ? nit : NS;
    for (int j = 0; j < n0; ++j) issue(j);
  }

  // queues: [0] p, [1] D_x p, [2] D_y p, [3] r, [4] D_x r, [5] D_y r
  float q[6][C::QL];
  float dq[2][C::DL];  // delayed in-plane sums: p_xx + p_yy - A p, A r
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int i = 0; i < C::QL; ++i) q[a][i] = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int i = 0; i < C::DL; ++i) dq[a][i] = 0.f;

  const size_t plane = d.plane();
  const int li = ty * C::TX + tx;  // index inside an interior tile
  // in-plane second derivatives and axis of the previous head plane, whose
  // cross term is finished one iteration later
  float pfxx[2] = {0.f, 0.f}, pfyy[2] = {0.f, 0.f}, phx = 0.f, phy = 0.f;
  bool phead = false;

#pragma unroll 1
  for (int j0 = 0; j0 < nit; j0 += U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u;
      if (j >= nit) break;  // uniform
      const int s = j % NS;
      const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((j / NS) & 1));
      // Also the point where every thread has finished iteration j-1 (its
      // stage reads and its D_y scratch writes).
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicOr(err, kErrWaitTimeout);
          for (int jj = j; jj <= issued_hi; ++jj)
            (void)mbar_wait_bounded(smem_u32(&bars[jj % NS]), (uint32_t)((jj / NS) & 1));
        }
        return;
      }
      if (tid == 0 && j >= 1 && j - 1 + NS < nit) issue(j - 1 + NS);

      // finish head plane j-1: D_x(D_y f) from scratch buffer (j-1)&1, then
      // its in-plane sums into the delay queue (slot R+u-1; for u = 0 that
      // is the previous group's last slot after the shift)
      if (!SH && j >= 1) {
        float a0 = 0.f, a1 = 0.f;
        if (phead) {
          float A[2];
#pragma unroll
          for (int f = 0; f < 2; ++f) {
            const float *sr = scr + (((j - 1) & 1) * 2 * C::TY + f * C::TY + ty) * C::SY + R + tx;
            float xy = 0.f;
#pragma unroll
            for (int m = 1; m <= R; ++m) xy = fmaf(w.c1[m], sr[m] - sr[-m], xy);
            A[f] = phx * phx * pfxx[f] + phy * phy * pfyy[f] + 2.f * phx * phy * xy;
          }
          a0 = pfxx[0] + pfyy[0] - A[0];
          a1 = A[1];
        }
        dq[0][R + u - 1] = a0;
        dq[1][R + u - 1] = a1;
      }

      const unsigned char *st = smem + s * C::STAGE_B;
      const int zh = z0 - R + j;
      const bool head = (zh >= 0 && zh < d.NZ);
      float *sb = scr + (j & 1) * 2 * C::TY * C::SY;
      if (head) {
        // shuffle variant: the head plane's axis and in-plane sums now
        float hx = 0.f, hy = 0.f, Ash[2] = {0.f, 0.f};
        if constexpr (SH) {
          const T *HA = (const T *)(st + 2 * C::HALO_B);
          hx = St<T>::ld(HA[li]);
          hy = St<T>::ld(HA[C::INT_B / C::EL + li]);
        }
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          const T *H = (const T *)(st + f * C::HALO_B);
          const T *row = H + (ty + R) * C::BXH + C::HX + tx;
          const float fc = St<T>::ld(row[0]);
          float xx = w.w2[0] * fc, yy = w.w2[0] * fc, dx = 0.f, dy = 0.f;
#pragma unroll
          for (int m = 1; m <= R; ++m) {
            const float xp = St<T>::ld(row[m]), xm = St<T>::ld(row[-m]);
            const float yp = St<T>::ld(row[m * C::BXH]), ym = St<T>::ld(row[-m * C::BXH]);
            xx = fmaf(w.w2[m], xp + xm, xx);
            dx = fmaf(w.c1[m], xp - xm, dx);
            yy = fmaf(w.w2[m], yp + ym, yy);
            dy = fmaf(w.c1[m], yp - ym, dy);
          }
          pfxx[f] = xx;
          pfyy[f] = yy;
          q[3 * f + 0][2 * R + u] = fc;
          q[3 * f + 1][2 * R + u] = dx;
          q[3 * f + 2][2 * R + u] = dy;
          if constexpr (SH) {
            // D_x(D_y f) by warp shuffles: the warp is one row of 32
            // points; lanes 0..R-1 also hold D_y f of the halo columns
            // x = -R..-1 and lanes R..2R-1 those of x = 32..32+R-1
            float dyh = 0.f;
            if (tx < 2 * R) {
              const int xo = tx < R ? tx - R : C::TX + (tx - R);
              const T *col = H + (ty + R) * C::BXH + C::HX + xo;
#pragma unroll
              for (int m = 1; m <= R; ++m)
                dyh = fmaf(w.c1[m], St<T>::ld(col[m * C::BXH]) - St<T>::ld(col[-m * C::BXH]), dyh);
            }
            float xy = 0.f;
#pragma unroll
            for (int m = 1; m <= R; ++m) {
              const int xp = tx + m, xm = tx - m;
              const float ap = __shfl_sync(0xffffffffu, dy, xp & 31);
              const float bp = __shfl_sync(0xffffffffu, dyh, (R + xp - C::TX) & 31);
              const float am = __shfl_sync(0xffffffffu, dy, xm & 31);
              const float bm = __shfl_sync(0xffffffffu, dyh, (xm + R) & 31);
              xy = fmaf(w.c1[m], (xp < C::TX ? ap : bp) - (xm >= 0 ? am : bm), xy);
            }
            Ash[f] = hx * hx * xx + hy * hy * yy + 2.f * hx * hy * xy;
          } else {
            sb[(f * C::TY + ty) * C::SY + R + tx] = dy;
          }
        }
        // D_y of both fields in the x halo columns [-R, 0) and [32, 32 + R):
        // HPW items per warp, one per lane
        if (!SH && tx < C::HPW) {
          const int t = ty * C::HPW + tx;
          if (t < C::NHALO) {
            const int f = t / (2 * R * C::TY);
            const int rem = t - f * (2 * R * C::TY);
            const int yy_ = rem / (2 * R);
            const int k = rem - yy_ * (2 * R);
            const int xo = k < R ? k - R : C::TX + (k - R);  // tile x of the halo column
            const T *H = (const T *)(st + f * C::HALO_B);
            const T *col = H + (yy_ + R) * C::BXH + C::HX + xo;
            float dy = 0.f;
#pragma unroll
            for (int m = 1; m <= R; ++m)
              dy = fmaf(w.c1[m], St<T>::ld(col[m * C::BXH]) - St<T>::ld(col[-m * C::BXH]), dy);
            sb[(f * C::TY + yy_) * C::SY + R + xo] = dy;
          }
        }
        if constexpr (SH) {
          dq[0][R + u] = pfxx[0] + pfyy[0] - Ash[0];
          dq[1][R + u] = Ash[1];
        } else {
          const T *HA = (const T *)(st + 2 * C::HALO_B);
          phx = St<T>::ld(HA[li]);
          phy = St<T>::ld(HA[C::INT_B / C::EL + li]);
        }
      } else {
#pragma unroll
        for (int a = 0; a < 6; ++a) q[a][2 * R + u] = 0.f;
        if constexpr (SH) {
          dq[0][R + u] = 0.f;
          dq[1][R + u] = 0.f;
        }
      }
      phead = head;
      if (j < 2 * R) continue;

      // output plane zo = zh - R
      const int zo = zh - R;
      const T *O = (const T *)(st + 2 * C::HALO_B);
      auto tileval = [&](int i) { return St<T>::ld(O[i * (C::INT_B / C::EL) + li]); };
      const float pm = tileval(2), rm = tileval(3), cc = tileval(4), ee = tileval(5), dd = tileval(6);
      const float nx = tileval(7), ny = tileval(8);
      const float nz = sqrtf(fmaxf(0.f, 1.f - nx * nx - ny * ny));
      float zz[2], xz[2], yz[2];
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        float a = w.w2[0] * q[3 * f][u + R], b = 0.f, c = 0.f;
#pragma unroll
        for (int m = 1; m <= R; ++m) {
          a = fmaf(w.w2[m], q[3 * f][u + R + m] + q[3 * f][u + R - m], a);
          b = fmaf(w.c1[m], q[3 * f + 1][u + R + m] - q[3 * f + 1][u + R - m], b);
          c = fmaf(w.c1[m], q[3 * f + 2][u + R + m] - q[3 * f + 2][u + R - m], c);
        }
        zz[f] = a;
        xz[f] = b;
        yz[f] = c;
      }
      const float Hp = dq[0][u] + (1.f - nz * nz) * zz[0] - 2.f * nz * (nx * xz[0] + ny * yz[0]);
      const float Gr = dq[1][u] + nz * nz * zz[1] + 2.f * nz * (nx * xz[1] + ny * yz[1]);
      const float gh = gxr + gyr + gzs[zo - z0];
      const float inv = __fdividef(1.f, 1.f + gh), qq = 1.f - gh;
      const float pn = (2.f * q[0][u + R] - qq * pm + cc * (ee * Hp + dd * Gr)) * inv;
      const float rn = (2.f * q[3][u + R] - qq * rm + cc * (dd * Hp + Gr)) * inv;
      const int x = x0 + tx, y = y0 + ty;
      if (x < d.NX && y < d.NY) {
        const size_t o = (size_t)zo * plane + (size_t)y * d.Xp + x;
        p_out[o] = St<T>::st(pn);
        r_out[o] = St<T>::st(rn);
      }
    }
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int i = 0; i < 2 * R; ++i) q[a][i] = q[a][i + U];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int i = 0; i < R; ++i) dq[a][i] = dq[a][i + U];
  }
}

// Field-pair variant of the kernel above (scratch cross term): p and r go
// through the same stencils with the same weights, so their arithmetic runs
// on (p, r) pairs with f32x2 instructions (__ffma2_rn, __fadd2_rn,
// __fmul2_rn; per component the scalar rounding), a difference a - b taken
// as c1 a + (-c1) b. Fewer issue slots, more registers: faster at orders up
// to 8, slower above (occupancy). With RY > 1 a thread owns RY consecutive
// rows of its column: the y taps of the rows overlap (2R + RY loads instead
// of RY (2R + 1)) and the per-plane work (ring wait, barrier, addressing,
// damping) is shared by RY points; each row's arithmetic is the RY = 1
// arithmetic, so the results are the same bits.
template <typename T, int R, int BY, int NS, int U, int RY = 1>
__global__ void __launch_bounds__(32 * BY)
    tti_tma_pk_kernel(const __grid_constant__ CUtensorMap m_ph, const __grid_constant__ CUtensorMap m_rh,
                      const __grid_constant__ CUtensorMap m_pm, const __grid_constant__ CUtensorMap m_rm,
                      const __grid_constant__ CUtensorMap m_c, const __grid_constant__ CUtensorMap m_e,
                      const __grid_constant__ CUtensorMap m_d, const __grid_constant__ CUtensorMap m_ax,
                      const __grid_constant__ CUtensorMap m_ay, T *__restrict__ p_out,
                      T *__restrict__ r_out, Dims d, Weights w, Sponge sp, int zc, int *err) {
  using C = TtiTile<T, R, BY, NS, U, false, RY>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  // [2][TY][SY] (D_y p, D_y r) pairs: one 8-byte load per cross-term tap
  float2 *scr = (float2 *)(smem + NS * C::STAGE_B);
  uint64_t *bars = (uint64_t *)(smem + NS * C::STAGE_B + C::SCR_B);
  float *gzs = (float *)(smem + NS * C::STAGE_B + C::SCR_B + C::BAR_B);

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int ry0 = ty * RY;  // first tile row of this thread
  const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, d.NZ);
  if (z0 >= z1 || zc > kMaxZChunk) return;  // uniform over the CTA
  const int nit = (z1 - z0) + 2 * R;
  const float gxr = (x0 + tx < d.NX) ? sp.gx[x0 + tx] : 0.f;
  float gyr[RY];
#pragma unroll
  for (int k = 0; k < RY; ++k) gyr[k] = (y0 + ry0 + k < d.NY) ? sp.gy[y0 + ry0 + k] : 0.f;

  const CUtensorMap *maps_int[C::N_INT] = {&m_ax, &m_ay, &m_pm, &m_rm, &m_c, &m_e, &m_d, &m_ax, &m_ay};
  if (tid == 0) {
    prefetch_tensormap(&m_ph);
    prefetch_tensormap(&m_rh);
#pragma unroll
    for (int i = 0; i < 7; ++i) prefetch_tensormap(maps_int[2 + i]);
#pragma unroll
    for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
    fence_barrier_init();
  }
  for (int i = tid; i < z1 - z0; i += C::THREADS) gzs[i] = sp.gz[z0 + i];
  __syncthreads();

  int issued_hi = -1;
  auto issue = [&](int j) {
    const int s = j % NS;
    const int zh = z0 - R + j;
    const bool head = (zh >= 0 && zh < d.NZ);
    const bool outp = (j >= 2 * R);
    const uint32_t bytes = (head ? (2 * C::BXH * C::BYH + 2 * C::TX * C::TY) * C::EL : 0) +
                           (outp ? 7 * C::TX * C::TY * C::EL : 0);
    const uint32_t bar = smem_u32(&bars[s]);
    unsigned char *st = smem + s * C::STAGE_B;
    mbar_arrive_expect_tx(bar, bytes);
    if (head) {
      tma_load_3d(smem_u32(st), &m_ph, x0 - C::HX, y0 - R, zh, bar);
      tma_load_3d(smem_u32(st + C::HALO_B), &m_rh, x0 - C::HX, y0 - R, zh, bar);
      tma_load_3d(smem_u32(st + 2 * C::HALO_B + 0 * C::INT_B), &m_ax, x0, y0, zh, bar);
      tma_load_3d(smem_u32(st + 2 * C::HALO_B + 1 * C::INT_B), &m_ay, x0, y0, zh, bar);
    }
    if (outp) {
      const int zo = zh - R;
#pragma unroll
      for (int i = 2; i < C::N_INT; ++i)
        tma_load_3d(smem_u32(st + 2 * C::HALO_B + i * C::INT_B), maps_int[i], x0, y0, zo, bar);
    }
    issued_hi = j;
  };
  if (tid == 0) {
    const int n0 = nit < NS ? nit : NS;
    for (int j = 0; j < n0; ++j) issue(j);
  }

  // queues of (p, r) pairs per row: [0] f, [1] D_x f, [2] D_y f
  float2 q[RY][3][C::QL];
  float2 dq[RY][C::DL];  // delayed in-plane sums (p_xx + p_yy - A p, A r)
#pragma unroll
  for (int k = 0; k < RY; ++k) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int i = 0; i < C::QL; ++i) q[k][a][i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < C::DL; ++i) dq[k][i] = make_float2(0.f, 0.f);
  }

  const size_t plane = d.plane();
  const int li = ry0 * C::TX + tx;  // index of the first row inside an interior tile
  // in-plane second derivatives and axis of the previous head plane, whose
  // cross term is finished one iteration later
  float2 pfxx[RY], pfyy[RY];
  float phx[RY], phy[RY];
#pragma unroll
  for (int k = 0; k < RY; ++k) {
    pfxx[k] = make_float2(0.f, 0.f);
    pfyy[k] = make_float2(0.f, 0.f);
    phx[k] = 0.f;
    phy[k] = 0.f;
  }
  bool phead = false;
  // A f = nx^2 f_xx + ny^2 f_yy + 2 nx ny f_xy for both fields, and the
  // in-plane sums (f_xx + f_yy - A f for p, A f for r)
  auto inplane = [&](float hx, float hy, float2 fxx, float2 fyy, float2 fxy) {
    const float2 A = __ffma2_rn(make_float2(2.f * hx * hy, 2.f * hx * hy), fxy,
                                __ffma2_rn(make_float2(hy * hy, hy * hy), fyy,
                                           __fmul2_rn(make_float2(hx * hx, hx * hx), fxx)));
    return make_float2(fxx.x + fyy.x - A.x, A.y);
  };

#pragma unroll 1
  for (int j0 = 0; j0 < nit; j0 += U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u;
      if (j >= nit) break;  // uniform
      const int s = j % NS;
      const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((j / NS) & 1));
      // Also the point where every thread has finished iteration j-1 (its
      // stage reads and its D_y scratch writes).
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicOr(err, kErrWaitTimeout);
          for (int jj = j; jj <= issued_hi; ++jj)
            (void)mbar_wait_bounded(smem_u32(&bars[jj % NS]), (uint32_t)((jj / NS) & 1));
        }
        return;
      }
      if (tid == 0 && j >= 1 && j - 1 + NS < nit) issue(j - 1 + NS);

      // finish head plane j-1: D_x(D_y f) from scratch buffer (j-1)&1, then
      // its in-plane sums into the delay queue (slot R+u-1; for u = 0 that
      // is the previous group's last slot after the shift)
      if (j >= 1) {
#pragma unroll
        for (int k = 0; k < RY; ++k) {
          float2 a = make_float2(0.f, 0.f);
          if (phead) {
            const float2 *sr = scr + (((j - 1) & 1) * C::TY + ry0 + k) * C::SY + R + tx;
            float2 xy = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 1; m <= R; ++m) {
              xy = __ffma2_rn(w.c1p[m], sr[m], xy);
              xy = __ffma2_rn(w.c1n[m], sr[-m], xy);
            }
            a = inplane(phx[k], phy[k], pfxx[k], pfyy[k], xy);
          }
          dq[k][R + u - 1] = a;
        }
      }

      const unsigned char *st = smem + s * C::STAGE_B;
      const int zh = z0 - R + j;
      const bool head = (zh >= 0 && zh < d.NZ);
      float2 *sb = scr + (j & 1) * C::TY * C::SY;
      if (head) {
        const T *Hp = (const T *)st;
        const T *Hr = (const T *)(st + C::HALO_B);
        const int o0 = (ry0 + R) * C::BXH + C::HX + tx;
        auto pr = [&](int o) { return make_float2(St<T>::ld(Hp[o]), St<T>::ld(Hr[o])); };
        // with RY > 1 the column at x over rows ry0 - R .. ry0 + RY - 1 + R
        // is loaded once for the RY rows' y taps
        float2 cv[RY > 1 ? 2 * R + RY : 1];
        if constexpr (RY > 1) {
#pragma unroll
          for (int i = 0; i < 2 * R + RY; ++i) cv[i] = pr(o0 + (i - R) * C::BXH);
        }
        auto col = [&](int k, int i) {  // row k + i of the column
          if constexpr (RY > 1)
            return cv[R + k + i];
          else
            return pr(o0 + i * C::BXH);
        };
#pragma unroll
        for (int k = 0; k < RY; ++k) {
          const int ob = o0 + k * C::BXH;
          const float2 fc = col(k, 0);
          float2 xx = __fmul2_rn(w.w2p[0], fc), yy = xx, dx = make_float2(0.f, 0.f), dy = dx;
#pragma unroll
          for (int m = 1; m <= R; ++m) {
            const float2 xp = pr(ob + m), xm = pr(ob - m);
            const float2 yp = col(k, m), ym = col(k, -m);
            xx = __ffma2_rn(w.w2p[m], __fadd2_rn(xp, xm), xx);
            dx = __ffma2_rn(w.c1n[m], xm, __ffma2_rn(w.c1p[m], xp, dx));
            yy = __ffma2_rn(w.w2p[m], __fadd2_rn(yp, ym), yy);
            dy = __ffma2_rn(w.c1n[m], ym, __ffma2_rn(w.c1p[m], yp, dy));
          }
          pfxx[k] = xx;
          pfyy[k] = yy;
          q[k][0][2 * R + u] = fc;
          q[k][1][2 * R + u] = dx;
          q[k][2][2 * R + u] = dy;
          sb[(ry0 + k) * C::SY + R + tx] = dy;
        }
        // D_y of both fields in the x halo columns [-R, 0) and
        // [32, 32 + R): HPW items per warp, spread over its lanes
#pragma unroll
        for (int i = 0; i < C::HPW; i += 32) {
          const int t = ty * C::HPW + i + tx;
          if (i + tx < C::HPW && t < C::NHALO) {
            const int f = t / (2 * R * C::TY);
            const int rem = t - f * (2 * R * C::TY);
            const int yy_ = rem / (2 * R);
            const int k = rem - yy_ * (2 * R);
            const int xo = k < R ? k - R : C::TX + (k - R);  // tile x of the halo column
            const T *H = (const T *)(st + f * C::HALO_B);
            const T *hc = H + (yy_ + R) * C::BXH + C::HX + xo;
            float dyh = 0.f;
#pragma unroll
            for (int m = 1; m <= R; ++m)
              dyh = fmaf(w.c1[m], St<T>::ld(hc[m * C::BXH]) - St<T>::ld(hc[-m * C::BXH]), dyh);
            reinterpret_cast<float *>(sb + yy_ * C::SY + R + xo)[f] = dyh;
          }
        }
        const T *HA = (const T *)(st + 2 * C::HALO_B);
#pragma unroll
        for (int k = 0; k < RY; ++k) {
          phx[k] = St<T>::ld(HA[li + k * C::TX]);
          phy[k] = St<T>::ld(HA[C::INT_B / C::EL + li + k * C::TX]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < RY; ++k)
#pragma unroll
          for (int a = 0; a < 3; ++a) q[k][a][2 * R + u] = make_float2(0.f, 0.f);
      }
      phead = head;
      if (j < 2 * R) continue;

      // output plane zo = zh - R
      const int zo = zh - R;
      const T *O = (const T *)(st + 2 * C::HALO_B);
      const float gzo = gzs[zo - z0];
#pragma unroll
      for (int k = 0; k < RY; ++k) {
        const int lk = li + k * C::TX;
        auto tileval = [&](int i) { return St<T>::ld(O[i * (C::INT_B / C::EL) + lk]); };
        const float pm = tileval(2), rm = tileval(3), cc = tileval(4), ee = tileval(5), dd = tileval(6);
        const float nx = tileval(7), ny = tileval(8);
        const float nz = sqrtf(fmaxf(0.f, 1.f - nx * nx - ny * ny));
        const float2 *f0 = q[k][0], *f1 = q[k][1], *f2 = q[k][2];
        float2 zz = __fmul2_rn(w.w2p[0], f0[u + R]), xz = make_float2(0.f, 0.f), yz = xz;
#pragma unroll
        for (int m = 1; m <= R; ++m) {
          zz = __ffma2_rn(w.w2p[m], __fadd2_rn(f0[u + R + m], f0[u + R - m]), zz);
          xz = __ffma2_rn(w.c1n[m], f1[u + R - m], __ffma2_rn(w.c1p[m], f1[u + R + m], xz));
          yz = __ffma2_rn(w.c1n[m], f2[u + R - m], __ffma2_rn(w.c1p[m], f2[u + R + m], yz));
        }
        const float Hp = dq[k][u].x + (1.f - nz * nz) * zz.x - 2.f * nz * (nx * xz.x + ny * yz.x);
        const float Gr = dq[k][u].y + nz * nz * zz.y + 2.f * nz * (nx * xz.y + ny * yz.y);
        const float gh = gxr + gyr[k] + gzo;
        const float inv = __fdividef(1.f, 1.f + gh), qq = 1.f - gh;
        const float pn = (2.f * f0[u + R].x - qq * pm + cc * (ee * Hp + dd * Gr)) * inv;
        const float rn = (2.f * f0[u + R].y - qq * rm + cc * (dd * Hp + Gr)) * inv;
        const int x = x0 + tx, y = y0 + ry0 + k;
        if (x < d.NX && y < d.NY) {
          const size_t o = (size_t)zo * plane + (size_t)y * d.Xp + x;
          p_out[o] = St<T>::st(pn);
          r_out[o] = St<T>::st(rn);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < RY; ++k) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) q[k][a][i] = q[k][a][i + U];
#pragma unroll
      for (int i = 0; i < R; ++i) dq[k][i] = dq[k][i + U];
    }
  }
}

}  // namespace fdw

namespace fdw {

constexpr int kTtiNS = 4;

// Candidate configurations (warps per CTA BY, z unrolling U, variant: 0
// scalar with the cross term through the shared D_y scratch, 1 scalar with
// warp shuffles, 2 field pairs with the scratch, 3 field pairs with two rows
// per thread), selected at run time by index. The shuffle form needs four
// shuffles per tap (interior and halo lane, both sides) where the scratch
// needs two shared loads, and measures 17-25% slower; it stays selectable.
// Variant 3 exists up to order 8 (radius 4): above it the two rows' z
// queues do not fit the registers.
#define FDW_TTI_CFGS(X) \
  X(0, 8, 2, 0)         \
  X(1, 4, 4, 0)         \
  X(2, 4, 2, 0)         \
  X(3, 2, 2, 0)         \
  X(4, 4, 1, 0)         \
  X(5, 4, 4, 1)         \
  X(6, 4, 2, 1)         \
  X(7, 4, 4, 2)         \
  X(8, 4, 1, 2)         \
  X(9, 4, 2, 3)         \
  X(10, 4, 1, 3)        \
  X(11, 2, 2, 3)        \
  X(12, 4, 4, 3)
constexpr int kTtiTiles = 13;
constexpr int kTtiRowPairMaxR = 4;

constexpr int tti_rows_per_thread(int V) { return V == 3 ? 2 : 1; }
template <int R, int V>
constexpr bool tti_cfg_exists() { return tti_rows_per_thread(V) == 1 || R <= kTtiRowPairMaxR; }

template <typename T, int R, int BY, int U, int V>
cudaError_t launch_tti_cfg_impl(const TTILaunch &L, cudaStream_t st) {
  using C = TtiTile<T, R, BY, kTtiNS, U, V == 1, tti_rows_per_thread(V)>;
  auto kern = [] {
    if constexpr (V >= 2)
      return tti_tma_pk_kernel<T, R, BY, kTtiNS, U, tti_rows_per_thread(V)>;
    else
      return tti_tma_kernel<T, R, BY, kTtiNS, U, V == 1>;
  }();
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
  kern<<<grd, blk, C::SMEM_B, st>>>(*L.m_ph, *L.m_rh, *L.m_pm, *L.m_rm, *L.m_c, *L.m_e, *L.m_d,
                                     *L.m_ax, *L.m_ay, (T *)L.p_prev, (T *)L.r_prev, L.d, L.w,
                                     L.sp, zc, L.err);
  return cudaGetLastError();
}

template <typename T, int R, int BY, int U, int V>
cudaError_t launch_tti_cfg(const TTILaunch &L, cudaStream_t st) {
  if constexpr (tti_cfg_exists<R, V>())
    return launch_tti_cfg_impl<T, R, BY, U, V>(L, st);
  else
    return cudaErrorInvalidValue;
}

template <typename T, int R, int BY, int U, int V>
int tti_geom_cfg(TileGeom *g) {
  if constexpr (!tti_cfg_exists<R, V>()) {
    return -1;
  } else {
    using C = TtiTile<T, R, BY, kTtiNS, U, V == 1, tti_rows_per_thread(V)>;
    g->box_halo_x = C::BXH;
    g->box_halo_y = C::BYH;
    g->box_int_x = C::TX;
    g->box_int_y = C::TY;
    g->smem = C::SMEM_B;
    return 0;
  }
}

#define FDW_TTI_CASE_LAUNCH(ID, BY, U, V) \
  case ID: return launch_tti_cfg<TYPE_, R, BY, U, V>(L, st);
#define FDW_TTI_CASE_GEOM(ID, BY, U, V) \
  case ID: return tti_geom_cfg<TYPE_, R, BY, U, V>(g);

#define FDW_TTI_DEFINE_STORAGE(SUFFIX, TYPE)                                  \
  template <typename TYPE_, int R>                                            \
  static cudaError_t tti_r_##SUFFIX(const TTILaunch &L, cudaStream_t st) {    \
    switch (L.tile) {                                                         \
      FDW_TTI_CFGS(FDW_TTI_CASE_LAUNCH)                                       \
      default: return cudaErrorInvalidValue;                                  \
    }                                                                         \
  }                                                                           \
  template <typename TYPE_, int R>                                            \
  static int tti_geom_r_##SUFFIX(int tile, TileGeom *g) {                     \
    switch (tile) {                                                           \
      FDW_TTI_CFGS(FDW_TTI_CASE_GEOM)                                         \
      default: return -1;                                                     \
    }                                                                         \
  }                                                                           \
  cudaError_t launch_tti_tma_##SUFFIX(const TTILaunch &L, cudaStream_t st) {  \
    switch (L.r) {                                                            \
      case 1: return tti_r_##SUFFIX<TYPE, 1>(L, st);                          \
      case 2: return tti_r_##SUFFIX<TYPE, 2>(L, st);                          \
      case 3: return tti_r_##SUFFIX<TYPE, 3>(L, st);                          \
      case 4: return tti_r_##SUFFIX<TYPE, 4>(L, st);                          \
      case 5: return tti_r_##SUFFIX<TYPE, 5>(L, st);                          \
      case 6: return tti_r_##SUFFIX<TYPE, 6>(L, st);                          \
      case 7: return tti_r_##SUFFIX<TYPE, 7>(L, st);                          \
      case 8: return tti_r_##SUFFIX<TYPE, 8>(L, st);                          \
      default: return cudaErrorInvalidValue;                                  \
    }                                                                         \
  }                                                                           \
  int tti_geom_##SUFFIX(int r, int tile, TileGeom *g) {                       \
    switch (r) {                                                              \
      case 1: return tti_geom_r_##SUFFIX<TYPE, 1>(tile, g);                   \
      case 2: return tti_geom_r_##SUFFIX<TYPE, 2>(tile, g);                   \
      case 3: return tti_geom_r_##SUFFIX<TYPE, 3>(tile, g);                   \
      case 4: return tti_geom_r_##SUFFIX<TYPE, 4>(tile, g);                   \
      case 5: return tti_geom_r_##SUFFIX<TYPE, 5>(tile, g);                   \
      case 6: return tti_geom_r_##SUFFIX<TYPE, 6>(tile, g);                   \
      case 7: return tti_geom_r_##SUFFIX<TYPE, 7>(tile, g);                   \
      case 8: return tti_geom_r_##SUFFIX<TYPE, 8>(tile, g);                   \
      default: return -1;                                                     \
    }                                                                         \
  }

}  // namespace fdw
