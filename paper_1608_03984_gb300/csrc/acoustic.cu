// acoustic.cu -- the acoustic time step (Algorithm 1 with Eq. Acou and the
// fused sponge) for sm_103a.
//
//   P u+ = 2u - Q u- + c lap_h(u),   c = (v dt / h)^2, P,Q = 1 +- gamma dt/2
//   lap_h(u) = sum over x, y, z of [w0 u + sum_{m=1..r} w_m (u_{+m} + u_{-m})]
//
// The star stencil of width k = 2r+1 per axis (Section "Stencil operators")
// reads u at 6r+1 points; the paper's byte count for it is 16 B per point
// (load u_n, u_{n-1}, the medium; store u_{n+1}, Table 1 / Eq. eqn_oi with
// l + s = 4 fields).
//
// Kernel design (2.5D z-march):
//   * a CTA owns a 32 x TY column of the grid and marches a chunk of z
//     planes; each thread owns RY points of one x column;
//   * the z neighbours live in a per-thread register queue of 2r+1 planes;
//   * the x/y neighbours come from a shared-memory halo tile of the current
//     plane, loaded by TMA;
//   * TMA keeps NS stages in flight, each an mbarrier-tracked slot holding:
//     the interior tile of plane z+r (fed to the queue), and the halo tile,
//     u_{n-1} tile and c tile of the output plane z;
//   * u_{n+1} is written straight from registers with coalesced 128-byte
//     row stores (full sectors: no read-for-ownership);
//   * the damping uses three 1D tables (no HBM traffic);
//   * every mbarrier wait is bounded; a CTA that gives up sets the error flag,
//     drains its own copies (bounded) and exits.
#include "fdw_internal.h"
#include "fdwave.h"
#include "ptx.cuh"

#include <string.h>

namespace fdw {

template <typename T, int R, int BY, int RY, int NS>
struct AcTile {
  static constexpr int TX = kTileX;
  static constexpr int TY = BY * RY;
  static constexpr int EL = (int)sizeof(T);
  static constexpr int XALIGN = 16 / EL;  // TMA: x * element size multiple of 16 B
  static constexpr int HX = ((R + XALIGN - 1) / XALIGN) * XALIGN;
  static constexpr int BXH = TX + 2 * HX;
  static constexpr int BYH = TY + 2 * R;
  static constexpr int a128(int b) { return (b + 127) / 128 * 128; }
  static constexpr int HALO_B = a128(BXH * BYH * EL);
  static constexpr int INT_B = a128(TX * TY * EL);
  static constexpr int STAGE_B = HALO_B + 3 * INT_B;  // halo | head | prev | c
  static constexpr int BAR_B = 128;
  static constexpr int SMEM_B = NS * STAGE_B + BAR_B + a128((TX + TY) * 4) + 128;
  static constexpr int THREADS = 32 * BY;
  static_assert(NS >= 2, "ring needs two stages");
  static_assert(BXH <= 256 && BYH <= 256 && TY <= 256, "TMA box dimension limit");
  static_assert((BXH * EL) % 16 == 0 && (TX * EL) % 16 == 0, "TMA inner box bytes");
  static_assert((HX * EL) % 16 == 0, "TMA x coordinate alignment");
};

// Tile configuration per radius: BY thread rows, RY points per thread.
template <int R> struct AcCfg {
  static constexpr int BY = 4, RY = 4, NS = 4;
};

template <typename T, int R, int BY, int RY, int NS>
__global__ void __launch_bounds__(32 * BY)
    acoustic_tma_kernel(const __grid_constant__ CUtensorMap m_halo,
                        const __grid_constant__ CUtensorMap m_head,
                        const __grid_constant__ CUtensorMap m_prev,
                        const __grid_constant__ CUtensorMap m_c, T *__restrict__ out, Dims d,
                        Weights w, Sponge sp, int zc, int *err) {
  using C = AcTile<T, R, BY, RY, NS>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem =
      (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  uint64_t *bars = (uint64_t *)(smem + NS * C::STAGE_B);
  float *gxs = (float *)(smem + NS * C::STAGE_B + C::BAR_B);
  float *gys = gxs + C::TX;

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, d.NZ);
  if (z0 >= z1) return;  // uniform over the CTA
  const int nit = (z1 - z0) + 2 * R;

  if (tid == 0) {
    prefetch_tensormap(&m_halo);
    prefetch_tensormap(&m_head);
    prefetch_tensormap(&m_prev);
    prefetch_tensormap(&m_c);
#pragma unroll
    for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
    fence_barrier_init();
  }
  for (int i = tid; i < C::TX; i += C::THREADS) gxs[i] = (x0 + i < d.NX) ? sp.gx[x0 + i] : 0.f;
  for (int i = tid; i < C::TY; i += C::THREADS) gys[i] = (y0 + i < d.NY) ? sp.gy[y0 + i] : 0.f;
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

  float q[RY][2 * R + 1];
#pragma unroll
  for (int ry = 0; ry < RY; ++ry)
#pragma unroll
    for (int i = 0; i < 2 * R + 1; ++i) q[ry][i] = 0.f;

  const float wc = 3.f * w.w2[0];
  const size_t plane = d.plane();

#pragma unroll 1
  for (int j = 0; j < nit; ++j) {
    const int s = j % NS;
    const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((j / NS) & 1));
    // Also the point where every thread has finished iteration j-1.
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(err, kErrWaitTimeout);
        for (int jj = j; jj <= issued_hi; ++jj)
          (void)mbar_wait_bounded(smem_u32(&bars[jj % NS]), (uint32_t)((jj / NS) & 1));
      }
      return;
    }
    if (tid == 0 && j >= 1 && j - 1 + NS < nit) issue(j - 1 + NS);

    const unsigned char *st = smem + s * C::STAGE_B;
    const int zh = z0 - R + j;
    const bool head = (zh >= 0 && zh < d.NZ);
    const T *hd = (const T *)(st + C::HALO_B);
#pragma unroll
    for (int ry = 0; ry < RY; ++ry) {
#pragma unroll
      for (int i = 0; i < 2 * R; ++i) q[ry][i] = q[ry][i + 1];
      q[ry][2 * R] = head ? St<T>::ld(hd[(ty * RY + ry) * C::TX + tx]) : 0.f;
    }
    if (j < 2 * R) continue;

    const int zo = zh - R;
    const T *H = (const T *)st;
    const T *PV = (const T *)(st + C::HALO_B + C::INT_B);
    const T *CC = (const T *)(st + C::HALO_B + 2 * C::INT_B);
    float col[RY + 2 * R];
#pragma unroll
    for (int i = 0; i < RY + 2 * R; ++i) col[i] = St<T>::ld(H[(ty * RY + i) * C::BXH + C::HX + tx]);
    const float ghz = __ldg(&sp.gz[zo]);
#pragma unroll
    for (int ry = 0; ry < RY; ++ry) {
      const int yl = ty * RY + ry;
      const T *row = H + (yl + R) * C::BXH + C::HX + tx;
      const float uc = col[ry + R];
      float lx = 0.f, ly = 0.f, lz = 0.f;
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        lx = fmaf(w.w2[m], St<T>::ld(row[m]) + St<T>::ld(row[-m]), lx);
        ly = fmaf(w.w2[m], col[ry + R + m] + col[ry + R - m], ly);
        lz = fmaf(w.w2[m], q[ry][R + m] + q[ry][R - m], lz);
      }
      const float lap = fmaf(wc, uc, lx + ly + lz);
      const float um = St<T>::ld(PV[yl * C::TX + tx]);
      const float cc = St<T>::ld(CC[yl * C::TX + tx]);
      const float gh = gxs[tx] + gys[yl] + ghz;
      const float up = (2.f * uc - (1.f - gh) * um + cc * lap) * __frcp_rn(1.f + gh);
      const int x = x0 + tx, y = y0 + yl;
      if (x < d.NX && y < d.NY) out[(size_t)zo * plane + (size_t)y * d.Xp + x] = St<T>::st(up);
    }
  }
}

// One thread per point, plain global loads with bounds checks: an
// independent GPU formulation of the same step for cross-checks.
template <typename T, int R>
__global__ void __launch_bounds__(256)
    acoustic_naive_kernel(const T *__restrict__ cur, T *__restrict__ prev,
                          const T *__restrict__ c, Dims d, Weights w, Sponge sp) {
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
  prev[p] = St<T>::st(up);
}

template <typename T, int R>
static cudaError_t launch_r(const AcousticLaunch &L, cudaStream_t st) {
  if (L.naive && !L.prepare_only) {
    dim3 blk(32, 8), grd((L.d.NX + 31) / 32, (L.d.NY + 7) / 8, L.d.NZ);
    acoustic_naive_kernel<T, R><<<grd, blk, 0, st>>>((const T *)L.cur, (T *)L.prev,
                                                     (const T *)L.c, L.d, L.w, L.sp);
    return cudaGetLastError();
  }
  using Cfg = AcCfg<R>;
  using C = AcTile<T, R, Cfg::BY, Cfg::RY, Cfg::NS>;
  auto kern = acoustic_tma_kernel<T, R, Cfg::BY, Cfg::RY, Cfg::NS>;
  if (L.prepare_only)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_B);
  const int zch = L.zchunks < 1 ? 1 : L.zchunks;
  const int zc = (L.d.NZ + zch - 1) / zch;
  dim3 grd((L.d.NX + C::TX - 1) / C::TX, (L.d.NY + C::TY - 1) / C::TY, (L.d.NZ + zc - 1) / zc);
  dim3 blk(32, Cfg::BY);
  kern<<<grd, blk, C::SMEM_B, st>>>(*L.map_cur_halo, *L.map_cur_int, *L.map_prev_int,
                                     *L.map_c_int, (T *)L.prev, L.d, L.w, L.sp, zc, L.err);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_t(const AcousticLaunch &L, cudaStream_t st) {
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

cudaError_t launch_acoustic(const AcousticLaunch &L, cudaStream_t st) {
  switch (L.storage) {
    case FDW_F32: return launch_t<float>(L, st);
    case FDW_BF16: return launch_t<__nv_bfloat16>(L, st);
    case FDW_F16: return launch_t<__half>(L, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t acoustic_prepare(int storage, int r) {
  AcousticLaunch L;
  memset(&L, 0, sizeof L);
  L.storage = storage;
  L.r = r;
  L.prepare_only = 1;
  return launch_acoustic(L, 0);
}

template <typename T, int R>
static void tile_r(int *bhx, int *bhy, int *bix, int *biy) {
  using Cfg = AcCfg<R>;
  using C = AcTile<T, R, Cfg::BY, Cfg::RY, Cfg::NS>;
  *bhx = C::BXH;
  *bhy = C::BYH;
  *bix = C::TX;
  *biy = C::TY;
}

template <typename T>
static void tile_t(int r, int *a, int *b, int *c, int *e) {
  switch (r) {
    case 1: tile_r<T, 1>(a, b, c, e); break;
    case 2: tile_r<T, 2>(a, b, c, e); break;
    case 3: tile_r<T, 3>(a, b, c, e); break;
    case 4: tile_r<T, 4>(a, b, c, e); break;
    case 5: tile_r<T, 5>(a, b, c, e); break;
    case 6: tile_r<T, 6>(a, b, c, e); break;
    case 7: tile_r<T, 7>(a, b, c, e); break;
    default: tile_r<T, 8>(a, b, c, e); break;
  }
}

void acoustic_tile(int storage, int r, int *bhx, int *bhy, int *bix, int *biy) {
  if (storage == FDW_F32) tile_t<float>(r, bhx, bhy, bix, biy);
  else if (storage == FDW_BF16) tile_t<__nv_bfloat16>(r, bhx, bhy, bix, biy);
  else tile_t<__half>(r, bhx, bhy, bix, biy);
}

}  // namespace fdw
