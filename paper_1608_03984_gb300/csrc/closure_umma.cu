// closure_umma.cu -- inference of the learned closure on the Blackwell
// tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// The network (closure.cu: three 3x3x3 convolutions 3 -> 16 -> 16 -> 1,
// ReLU between, zero padding at the faces of the grid) runs over the box of
// points the time loop corrects, in one persistent kernel: each CTA takes
// work items (an output column of TXO x TYO points and a chunk of z planes,
// tiling the box) and marches the planes through
// a pipeline whose three convolutions are implicit GEMMs with
//   M = 128 points (an 8 x 16 block of one plane; the 8-row core matrices
//       of the operand are 8 consecutive x points, stepped by the row
//       stride of the plane, so a tap's in-plane shift (dy, dx) is only a
//       shift of the operand's start address by dy rows + dx points),
//   K = 16 (FP16 channels),
//   N = 3 x 16: the three z taps of a layer share each operand read -- an
//       input plane adds to the accumulators of the three output planes it
//       touches (z - 1, z, z + 1), which live side by side in tensor memory
//       as 16-column slots; the weights' column blocks are permuted per
//       plane (three phases) so that slot j always holds the plane = j mod 3.
// Layer 1 has 3 real input channels, so its K packs (y - 1, y, y + 1) x 4
// channels (an input plane is stored "y-stacked") and the x taps are
// operand shifts: 3 MMAs per block and plane. Layer 2: 9 MMAs (the in-plane
// taps). Layer 3 has one output channel: M = 128 points, N = 32 (the 27
// taps, padded) gives every tap's product at every point, and a gather sums
// the 27 products of each output point (fixed order: deterministic).
//
// Roles (512 threads, one CTA per SM; every wait is bounded):
//   warps 0, 1, 3  stack the next input plane (FP16 x = (u/s, u_{n-1}/s, v',
//                  0)) into shared memory;
//   warp 2         allocates the 512 tensor-memory columns, runs the MMA
//                  schedule (one elected lane issues the MMAs and commits
//                  them to mbarriers);
//   warps 4-7      epilogue of layer 1, warps 12-15 that of layer 2:
//                  tcgen05.ld of a completed plane's slot, bias, ReLU, zero
//                  outside the grid, FP16 into the next layer's operand,
//                  the slot cleared;
//   warps 8-11     layer-3 products out of tensor memory, the gather, the
//                  output planes.
// Issue order per plane s: layer 1 of plane s + 1, layer 3 of plane s - 1,
// layer 2 of plane s -- so the tensor core has work while an epilogue
// drains the accumulators the next group needs.
#include <math.h>
#include <stdint.h>

#include "fdw_internal.h"
#include "fdwave.h"
#include "ptx.cuh"

namespace fdw {

namespace um {

constexpr int TXO = 12, TYO = 28;  // output points of a work item per plane
constexpr int NOUT = TXO * TYO;
// Arrays of one plane (CTA-local coordinates, output tile at [0, TXO) x [0, TYO)):
//   X  (stacked input): x in [-3, 15), y in [-2, 30)
//   A1 (layer-1 output): x in [-2, 16), y in [-2, 32)  (layer 1 writes [-2,14) x [-2,30))
//   A2 (layer-2 output): x in [-1, 17), y in [-1, 31)  (layer 2 writes [-1,15) x [-1,31))
// each as two K halves (channels 0-7 | 8-15) of 16 bytes per point.
constexpr int XW = 18, XH = 32, A1W = 18, A1H = 34, A2W = 18, A2H = 32;
constexpr int X_HALF = XW * XH * 16, X_BUF = 2 * X_HALF;
constexpr int A1_HALF = A1W * A1H * 16, A1_BUF = 2 * A1_HALF;
constexpr int A2_HALF = A2W * A2H * 16, A2_BUF = 2 * A2_HALF;
constexpr int NP3 = 9;                    // layer-3 products per point: (dz, dy) taps, x summed
constexpr int D3_B = 4 * NP3 * 128 * 4;   // layer-3 products [block][(a, b)][point] FP32
constexpr int PEND_B = 3 * NOUT * 4;      // three pending output planes FP32
constexpr int BMAT = 48 * 16 * 2;         // one N = 48, K = 16 FP16 operand
constexpr int B1_B = 3 * 3 * BMAT;        // [phase][dx]
constexpr int B2_B = 3 * 9 * BMAT;        // [phase][dy * 3 + dx]
constexpr int B3_B = 3 * 16 * 16 * 2;     // [dx][n = a 3 + b][ci]
constexpr int OFF_X = 0;
constexpr int OFF_A1 = OFF_X + 2 * X_BUF;
constexpr int OFF_A2 = OFF_A1 + 2 * A1_BUF;
constexpr int OFF_D3 = OFF_A2 + A2_BUF;
constexpr int OFF_PEND = OFF_D3 + D3_B;
constexpr int OFF_B1 = OFF_PEND + PEND_B;
constexpr int OFF_B2 = OFF_B1 + B1_B;
constexpr int OFF_B3 = OFF_B2 + B2_B;
constexpr int OFF_BIAS = OFF_B3 + B3_B;   // b1[16], b2[16], b3, 2^-e3
constexpr int OFF_BAR = OFF_BIAS + 256;
constexpr int NBAR = 14;
constexpr int OFF_TSLOT = OFF_BAR + NBAR * 8;
constexpr int SMEM_USED = OFF_TSLOT + 16;
constexpr int SMEM_B = SMEM_USED + 128;   // + alignment of the dynamic base
static_assert(SMEM_B <= 227 * 1024, "shared memory per CTA");
// tcgen05 operands without swizzle need 16-byte aligned starts
static_assert(OFF_A1 % 16 == 0 && OFF_A2 % 16 == 0 && OFF_D3 % 16 == 0 && OFF_B1 % 16 == 0 &&
                  OFF_B2 % 16 == 0 && OFF_B3 % 16 == 0 && OFF_BAR % 8 == 0,
              "operand alignment");
// tensor-memory columns: layer-1 slots, layer-2 slots (48 per block), layer-3 products (32 per block)
constexpr uint32_t TM_L1 = 0, TM_L2 = 192, TM_L3 = 384, TM_COLS = 512;  // layer 3: 16 per block
constexpr int NTHR = 512;
constexpr int NLOAD = 96;  // threads of the stacking warps 0, 1, 3
// mbarriers
enum {
  BAR_XFULL0 = 0, BAR_XFULL1, BAR_L1_0, BAR_L1_1, BAR_E1, BAR_L2, BAR_A1F0, BAR_A1F1, BAR_E2, BAR_L3, BAR_E3,
  BAR_Z1, BAR_Z2, BAR_FINAL
};
// Each barrier completes once per event and its waiters consume every
// completion in order, at most one phase behind: the per-item clearing of
// the layer-1/2 slots has barriers of its own (BAR_Z1, BAR_Z2) so that an
// epilogue group's last arrival of an item and its clearing for the next
// item never land on the same barrier back to back.

}  // namespace um

// Operands of the tensor-core kernel in their shared-memory layout (each
// N x 16 matrix as its channel 0-7 half then its channel 8-15 half).
struct UmmaWeights {
  __half b1[3 * 3 * 48 * 16];  // [phase][dx][n = slot * 16 + co][k = dy * 4 + ci]
  __half b2[3 * 9 * 48 * 16];  // [phase][dy * 3 + dx][n][k = ci]
  __half b3[3 * 16 * 16];      // [dx c][n = a 3 + b][ci], times 2^e3; n >= 9 zero
  float b1f[16], b2f[16], b3f, w3_unscale;
};

namespace umx {

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // shared-memory matrix descriptor: start, leading (K) and stride (M/N)
  // byte offsets in 16-byte units, descriptor version 1, no swizzle
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulators, FP16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
// The issuing warp runs its loop with all 32 lanes (warp-uniform values stay
// in uniform registers); elect.sync picks the one lane that issues.
__device__ __forceinline__ void mma_elect(uint32_t d, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n.reg .pred e, p;\nelect.sync _|e, 0xffffffff;\nsetp.ne.b32 p, %4, 0;\n"
      "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit_elect(uint32_t bar) {
  asm volatile(
      "{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\n"
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// OR of v over the `n` threads of named barrier `id` (also a barrier)
__device__ __forceinline__ bool bar_or(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbar.red.or.pred p, %2, %3, q;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// 16 consecutive FP32 columns of this warp's 32 lanes
__device__ __forceinline__ void ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void st16_zero(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}

}  // namespace umx

// ---------------------------------------------------------------------------
// operand preparation (one block): the BF16 parameters (exact in FP16) in the
// kernel's layouts. Parameter order of the closure network (closure.cu):
// W1[co][ci][tap], b1, W2[co][ci][tap], b2, W3[ci][tap], b3, tap = a 9 + b 3
// + c for the offset (a - 1, b - 1, c - 1) in (z, y, x).
// ---------------------------------------------------------------------------
namespace umx {

// K-major operand element (n, k) of an N x 16 matrix stored as two halves
__device__ __forceinline__ int kidx(int N, int n, int k) { return (k >> 3) * N * 8 + n * 8 + (k & 7); }

// z tap a of the slot j block at phase phi: the input plane z adds to output
// plane p = z + rel with p = j (mod 3); the tap is a = 1 - rel
__device__ __forceinline__ int slot_tap(int phi, int j) {
  const int dl = ((j - phi) % 3 + 3) % 3;
  const int rel = dl <= 1 ? dl : -1;
  return 1 - rel;
}

}  // namespace umx

__global__ void umma_prepare_kernel(const __nv_bfloat16 *__restrict__ pb, const float *__restrict__ pf,
                                    UmmaWeights *__restrict__ w) {
  constexpr int H = 16;
  constexpr int OW1 = 0, OB1 = H * 3 * 27, OW2 = OB1 + H, OB2 = OW2 + H * H * 27, OW3 = OB2 + H,
                OB3 = OW3 + H * 27;
  __shared__ float amax[256];
  const int t = threadIdx.x;
  float m = 0.f;
  for (int i = t; i < H * 27; i += blockDim.x) m = fmaxf(m, fabsf(__bfloat162float(pb[OW3 + i])));
  amax[t] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s) amax[t] = fmaxf(amax[t], amax[t + s]);
    __syncthreads();
  }
  // 2^e3 max|W3| in [1, 2): exact scaling of the last layer into FP16's normal range
  const int e3 = amax[0] > 0.f ? -ilogbf(amax[0]) : 0;
  // layer 1: [phase][dx c][n = j 16 + co][k = b 4 + ci] (b = dy index, 3 = padding; ci = 3 padding)
  for (int i = t; i < 3 * 3 * 48 * 16; i += blockDim.x) {
    const int mat = i / (48 * 16), e = i % (48 * 16), n = e / 16, k = e % 16;
    const int phi = mat / 3, c = mat % 3, j = n / 16, co = n % 16, b = k / 4, ci = k % 4;
    float v = 0.f;
    if (b < 3 && ci < 3) {
      const int a = umx::slot_tap(phi, j);
      v = __bfloat162float(pb[OW1 + (co * 3 + ci) * 27 + a * 9 + b * 3 + c]);
    }
    w->b1[mat * 48 * 16 + umx::kidx(48, n, k)] = __float2half_rn(v);
  }
  // layer 2: [phase][b 3 + c][n = j 16 + co][k = ci]
  for (int i = t; i < 3 * 9 * 48 * 16; i += blockDim.x) {
    const int mat = i / (48 * 16), e = i % (48 * 16), n = e / 16, ci = e % 16;
    const int phi = mat / 9, bc = mat % 9, j = n / 16, co = n % 16;
    const int a = umx::slot_tap(phi, j);
    const float v = __bfloat162float(pb[OW2 + (co * H + ci) * 27 + a * 9 + bc]);
    w->b2[mat * 48 * 16 + umx::kidx(48, n, ci)] = __float2half_rn(v);
  }
  // layer 3: [dx c][n = a 3 + b][ci] times 2^e3 (the x taps are operand shifts)
  for (int i = t; i < 3 * 16 * 16; i += blockDim.x) {
    const int c = i / 256, n = (i / 16) % 16, ci = i % 16;
    const float v = n < 9 ? ldexpf(__bfloat162float(pb[OW3 + ci * 27 + n * 3 + c]), e3) : 0.f;
    w->b3[c * 256 + umx::kidx(16, n, ci)] = __float2half_rn(v);
  }
  if (t < 16) {
    w->b1f[t] = pf[OB1 + t];
    w->b2f[t] = pf[OB2 + t];
  }
  if (t == 0) {
    w->b3f = pf[OB3];
    w->w3_unscale = ldexpf(1.f, -e3);
  }
}

// ---------------------------------------------------------------------------
// the fused network kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(um::NTHR, 1)
    closure_umma_kernel(const uint2 *__restrict__ x16, const UmmaWeights *__restrict__ wg, float *__restrict__ out,
                        int NX, int NY, int NZ, int ox, int oy, int oz, int zend, int tiles_x, int tiles_y,
                        int zc, int nitems, int *err) {
  using namespace um;
  using namespace umx;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t *bars = (uint64_t *)(sm + OFF_BAR);
  volatile int *abort_flag = (volatile int *)(sm + OFF_TSLOT + 4);
  float *bias = (float *)(sm + OFF_BIAS);
  auto bar = [&](int i) { return smem_u32(&bars[i]); };
  // bounded wait on phase `parity` of barrier i; false (and the CTA told to
  // stop) after the time limit or once another role has given up
  auto wait = [&](int i, uint32_t parity) -> bool {
    if (*abort_flag) return false;
    if (mbar_wait_bounded(bar(i), parity)) return true;
    atomicOr(err, kErrWaitTimeout);
    *abort_flag = 1;
    return false;
  };

  // ---- set-up: operands, biases, zeroed layer-1 arrays, barriers, tensor memory
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(wg->b1);  // b1 | b2 | b3 are contiguous
    uint4 *dst = reinterpret_cast<uint4 *>(sm + OFF_B1);
    for (int i = tid; i < (B1_B + B2_B + B3_B) / 16; i += NTHR) dst[i] = src[i];
    if (tid < 16) {
      bias[tid] = wg->b1f[tid];
      bias[16 + tid] = wg->b2f[tid];
    }
    if (tid == 0) {
      bias[32] = wg->b3f;
      bias[33] = wg->w3_unscale;
    }
    uint4 *a1 = reinterpret_cast<uint4 *>(sm + OFF_A1);  // the margins of A1 and A2 stay zero
    for (int i = tid; i < (2 * A1_BUF + A2_BUF) / 16; i += NTHR) a1[i] = make_uint4(0u, 0u, 0u, 0u);
    float *pend = reinterpret_cast<float *>(sm + OFF_PEND);
    for (int i = tid; i < 3 * NOUT; i += NTHR) pend[i] = 0.f;
    if (tid == 0) {
      mbar_init(bar(BAR_XFULL0), NLOAD);
      mbar_init(bar(BAR_XFULL1), NLOAD);
      mbar_init(bar(BAR_L1_0), 1);
      mbar_init(bar(BAR_L1_1), 1);
      mbar_init(bar(BAR_E1), 128);
      mbar_init(bar(BAR_L2), 1);
      mbar_init(bar(BAR_A1F0), 1);
      mbar_init(bar(BAR_A1F1), 1);
      mbar_init(bar(BAR_E2), 128);
      mbar_init(bar(BAR_L3), 1);
      mbar_init(bar(BAR_E3), 128);
      mbar_init(bar(BAR_Z1), 128);
      mbar_init(bar(BAR_Z2), 128);
      mbar_init(bar(BAR_FINAL), 1);
      *abort_flag = 0;
      fence_barrier_init();
    }
    if (warp == 2) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(sm + OFF_TSLOT)),
                   "r"(TM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
  }
  const uint32_t tmem = *(volatile uint32_t *)(sm + OFF_TSLOT);
  const int tiles = tiles_x * tiles_y;
  auto mod3 = [](int v) { return ((v % 3) + 3) % 3; };

  if (warp == 0 || warp == 1 || warp == 3) {
    // ---- stacking warps: x planes into the y-stacked layer-1 operand; each
    // thread holds its points' next plane in registers (loaded one plane
    // ahead, so the global latency overlaps the wait for a free buffer)
    constexpr int PPT = XW * XH / NLOAD;  // points per thread
    static_assert(XW * XH == PPT * NLOAD, "stacking split");
    const int lt = (warp == 3 ? 64 : warp * 32) + lane;
    uint32_t fills = 0;
    uint2 pv[PPT][3];
    int X0 = 0, Y0 = 0;
    auto fetch = [&](int zi) {
      const bool zin = zi >= 0 && zi < NZ;
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        const int pt = lt + i * NLOAD;
        const int x = X0 - 3 + pt % XW, y = Y0 - 2 + pt / XW;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int yy = y - 1 + r;
          pv[i][r] = (zin && x >= 0 && x < NX && yy >= 0 && yy < NY)
                         ? x16[((size_t)zi * NY + yy) * NX + x]
                         : make_uint2(0u, 0u);
        }
      }
    };
    for (int item = blockIdx.x; item < nitems && !*abort_flag; item += gridDim.x) {
      const int tt = item % tiles, zk = item / tiles;
      X0 = ox + (tt % tiles_x) * TXO;
      Y0 = oy + (tt / tiles_x) * TYO;
      const int z0 = oz + zk * zc, z1 = min(z0 + zc, zend), nit = z1 - z0 + 6;
      fetch(z0 - 3);
      for (int s = 0; s < nit; ++s) {
        const int b = fills & 1;
        const uint32_t use = fills >> 1;
        if (use >= 1 && !wait(BAR_L1_0 + b, (use - 1) & 1)) break;  // layer 1 read this buffer
        uint4 *H0 = reinterpret_cast<uint4 *>(sm + OFF_X + b * X_BUF);
        uint4 *H1 = reinterpret_cast<uint4 *>(sm + OFF_X + b * X_BUF + X_HALF);
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          const int pt = lt + i * NLOAD;
          H0[pt] = make_uint4(pv[i][0].x, pv[i][0].y, pv[i][1].x, pv[i][1].y);
          H1[pt] = make_uint4(pv[i][2].x, pv[i][2].y, 0u, 0u);
        }
        fence_async_smem();
        mbar_arrive(bar(BAR_XFULL0 + b));
        ++fills;
        if (s + 1 < nit) fetch(z0 - 2 + s);
      }
    }
  } else if (warp == 2) {
    // ---- MMA issue: the whole warp runs the loop, one elected lane issues
    {
      uint32_t g1 = 0, g2 = 0, ge1 = 0, ge2 = 0, ge3 = 0, n3 = 0, gz = 0;
      const uint32_t id48 = idesc(128, 48), id16 = idesc(128, 16);
      // descriptors of every operand base; a tap's shift adds its 16-byte
      // offset to the start-address field (no carry: the field holds the
      // whole shared window)
      const uint64_t dX0 = sdesc(smem_u32(sm + OFF_X), X_HALF, XW * 16);
      const uint64_t dX1 = sdesc(smem_u32(sm + OFF_X + X_BUF), X_HALF, XW * 16);
      const uint64_t dA10 = sdesc(smem_u32(sm + OFF_A1), A1_HALF, A1W * 16);
      const uint64_t dA11 = sdesc(smem_u32(sm + OFF_A1 + A1_BUF), A1_HALF, A1W * 16);
      const uint64_t dA2 = sdesc(smem_u32(sm + OFF_A2), A2_HALF, A2W * 16);
      const uint64_t dB1 = sdesc(smem_u32(sm + OFF_B1), 48 * 16, 128);
      const uint64_t dB2 = sdesc(smem_u32(sm + OFF_B2), 48 * 16, 128);
      const uint64_t dB3 = sdesc(smem_u32(sm + OFF_B3), 16 * 16, 128);
      constexpr uint64_t kBM = BMAT / 16;  // one B matrix in 16-byte units
      bool ok = true;
      auto uwait = [&](int i, uint32_t parity) { return __all_sync(0xffffffffu, wait(i, parity)); };
      auto L1 = [&](int zi) -> bool {
        const int b = g1 & 1;
        if (!uwait(BAR_XFULL0 + b, (g1 >> 1) & 1)) return false;
        fence_after();
        const uint64_t a0 = b ? dX1 : dX0, b0 = dB1 + (uint64_t)mod3(zi) * 3 * kBM;
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            mma_elect(tmem + TM_L1 + 48 * k, a0 + (uint64_t)((16 * (k >> 1)) * XW + 8 * (k & 1) + c), b0 + c * kBM,
                id48, 1);
        commit_elect(bar(BAR_L1_0 + b));
        ++g1;
        return true;
      };
      auto L2 = [&](int p1) {
        const int b = g2 & 1;
        const uint64_t a0 = b ? dA11 : dA10, b0 = dB2 + (uint64_t)mod3(p1) * 9 * kBM;
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int t9 = 0; t9 < 9; ++t9)
            mma_elect(tmem + TM_L2 + 48 * k, a0 + (uint64_t)((16 * (k >> 1) + t9 / 3) * A1W + 8 * (k & 1) + t9 % 3),
                b0 + t9 * kBM, id48, 1);
        commit_elect(bar(BAR_L2));
        commit_elect(bar(BAR_A1F0 + b));  // layer 1 may refill this operand buffer
        ++g2;
      };
      auto L3 = [&]() -> bool {
        if (!uwait(BAR_E2, ge2++ & 1)) return false;           // a2 plane written, layer-2 slot cleared
        if (n3 >= 1 && !uwait(BAR_E3, ge3++ & 1)) return false;  // products of the previous plane taken
        fence_after();
        // block k covers output columns x in [8 kx, 8 kx + 8), rows y in
        // [-1 + 16 ky, 15 + 16 ky); the x tap c is an operand shift
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            mma_elect(tmem + TM_L3 + 16 * k, dA2 + (uint64_t)((16 * (k >> 1)) * A2W + 8 * (k & 1) + c),
                dB3 + (uint64_t)c * (256 * 2 / 16), id16, c > 0);
        commit_elect(bar(BAR_L3));
        ++n3;
        return true;
      };
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const int zk = item / tiles;
        const int z0 = oz + zk * zc, z1 = min(z0 + zc, zend), nit = z1 - z0 + 6;
        // tensor memory cleared for the item (layer-1 and layer-2 slots)
        ok = uwait(BAR_Z1, gz & 1) && uwait(BAR_Z2, gz & 1) && L1(z0 - 3);
        ++gz;
        for (int s = 0; s < nit && ok; ++s) {
          if (s + 1 < nit) ok = uwait(BAR_E1, ge1++ & 1) && L1(z0 - 2 + s);  // E1(s): slot cleared, a1 written
          if (ok && s >= 1) ok = L3();
          if (ok && s + 1 == nit) ok = uwait(BAR_E1, ge1++ & 1);
          if (ok) {
            fence_after();
            L2(z0 - 4 + s);
          }
        }
        if (ok) ok = L3();
      }
      // every MMA issued has completed before the tensor memory is freed
      commit_elect(bar(BAR_FINAL));
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar(BAR_FINAL), 0)) && lane == 0)
        atomicOr(err, kErrWaitTimeout);
    }
  } else if (warp < 8 || warp >= 12) {
    // ---- epilogues: warps 4-7 layer 1, warps 12-15 layer 2. A completed
    // plane's slot is read out of tensor memory (bias, ReLU, zero outside
    // the grid, FP16) into the next layer's operand, and cleared. Every
    // tcgen05.ld/st runs with the whole warp, so the decisions to go on are
    // made warp-uniform.
    const bool l1 = warp < 8;
    const int t = tid & 127;  // tensor-memory lane = M row of a block
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    const int px = t & 7, py = t >> 3;
    const uint32_t tm0 = l1 ? TM_L1 : TM_L2;
    const float *bs = bias + (l1 ? 0 : 16);
    uint32_t gl = 0;  // completions of this layer's MMA groups consumed
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
      const int tt = item % tiles, zk = item / tiles;
      const int X0 = ox + (tt % tiles_x) * TXO, Y0 = oy + (tt / tiles_x) * TYO;
      const int z0 = oz + zk * zc, z1 = min(z0 + zc, zend), nit = z1 - z0 + 6;
      for (uint32_t col = 0; col < 192; col += 16) st16_zero(tmem + lanes + tm0 + col);
      wait_st();
      fence_before();
      mbar_arrive(bar(l1 ? BAR_Z1 : BAR_Z2));
      bool ok = true;
      for (int s = 0; s < nit && ok; ++s) {
        unsigned char *dstb;
        int plane, ox, oy, W, HALF;
        if (l1) {
          // a1 plane z0 - 4 + s, complete after layer 1 of input plane z0 - 3 + s;
          // its operand buffer must have been read by layer 2 two planes ago
          const int b = gl & 1;
          ok = __all_sync(0xffffffffu, wait(BAR_L1_0 + b, (gl >> 1) & 1) &&
                                           (gl < 2 || wait(BAR_A1F0 + b, ((gl - 2) >> 1) & 1)));
          plane = z0 - 4 + s;
          dstb = sm + OFF_A1 + b * A1_BUF;
          ox = -2;
          oy = -2;
          W = A1W;
          HALF = A1_HALF;
        } else {
          // a2 plane z0 - 5 + s, complete after layer 2 of a1 plane z0 - 4 + s
          // (which also ends layer 3 of the previous plane: A2 is free)
          ok = __all_sync(0xffffffffu, wait(BAR_L2, gl & 1));
          plane = z0 - 5 + s;
          dstb = sm + OFF_A2;
          ox = -1;
          oy = -1;
          W = A2W;
          HALF = A2_HALF;
        }
        if (!ok) break;
        ++gl;
        fence_after();
        const uint32_t slot = tm0 + 16 * mod3(plane);
        const bool zin = plane >= 0 && plane < NZ;
#pragma unroll
        for (int kk = 0; kk < 4; kk += 2) {
          float v[2][16];
          ld16(tmem + lanes + slot + 48 * kk, v[0]);
          ld16(tmem + lanes + slot + 48 * (kk + 1), v[1]);
          wait_ld();
          st16_zero(tmem + lanes + slot + 48 * kk);
          st16_zero(tmem + lanes + slot + 48 * (kk + 1));
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int k = kk + h;
            const int x = ox + 8 * (k & 1) + px, y = oy + 16 * (k >> 1) + py;
            const int gx = X0 + x, gy = Y0 + y;
            const bool in = zin && gx >= 0 && gx < NX && gy >= 0 && gy < NY;
            uint32_t hv[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              __half2 hh = __floats2half2_rn(in ? fmaxf(v[h][2 * c] + bs[2 * c], 0.f) : 0.f,
                                             in ? fmaxf(v[h][2 * c + 1] + bs[2 * c + 1], 0.f) : 0.f);
              hv[c] = *reinterpret_cast<uint32_t *>(&hh);
            }
            const int idx = (y - oy) * W + (x - ox);
            *reinterpret_cast<uint4 *>(dstb + 16 * idx) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
            *reinterpret_cast<uint4 *>(dstb + HALF + 16 * idx) = make_uint4(hv[4], hv[5], hv[6], hv[7]);
          }
        }
        wait_st();
        fence_async_smem();
        fence_before();
        mbar_arrive(bar(l1 ? BAR_E1 : BAR_E2));
      }
      if (!ok) break;
    }
  } else {
    // ---- layer-3 products, gather, output planes
    const int wl = warp - 8, t = tid - 256;
    const uint32_t lanes = (uint32_t)(32 * wl) << 16;
    float *D3 = reinterpret_cast<float *>(sm + OFF_D3);
    float *pend = reinterpret_cast<float *>(sm + OFF_PEND);
    uint32_t gl3 = 0;
    bool stop = false;  // uniform over the four warps (decided through named barrier 1)
    // D3 index of product (0, b) for each output point of this thread
    // (product (a, b) adds a * 3 * 128): block and lane of the point
    // (ox, oy + b - 1), in layer-3 block coordinates (x from 0, y from -1)
    constexpr int JPT = (NOUT + 127) / 128;
    int gofs[JPT][3];
#pragma unroll
    for (int i = 0; i < JPT; ++i) {
      const int jo = t + 128 * i < NOUT ? t + 128 * i : 0;
      const int ox = jo % TXO, oy = jo / TXO;
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        const int qy = oy + bb;
        const int k = (qy >> 4) * 2 + (ox >> 3), ln = (qy & 15) * 8 + (ox & 7);
        gofs[i][bb] = (k * NP3 + bb) * 128 + ln;
      }
    }
    for (int item = blockIdx.x; item < nitems && !stop; item += gridDim.x) {
      const int tt = item % tiles, zk = item / tiles;
      const int X0 = ox + (tt % tiles_x) * TXO, Y0 = oy + (tt / tiles_x) * TYO;
      const int z0 = oz + zk * zc, z1 = min(z0 + zc, zend), nit = z1 - z0 + 6;
      for (int s = 0; s < nit; ++s) {
        const bool ok = wait(BAR_L3, gl3 & 1);
        // one decision for the warpgroup; also the point where the previous
        // gather is done with D3
        if ((stop = bar_or(1, 128, !ok))) break;
        ++gl3;
        fence_after();
        {
          float v[4][16];
#pragma unroll
          for (int k = 0; k < 4; ++k) ld16(tmem + lanes + TM_L3 + 16 * k, v[k]);
          wait_ld();
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int n = 0; n < NP3; ++n) D3[(k * NP3 + n) * 128 + t] = v[k][n];
        }
        fence_before();
        mbar_arrive(bar(BAR_E3));
        asm volatile("bar.sync 1, 128;" ::: "memory");  // D3 complete
        const int p2 = z0 - 5 + s, zd = p2 - 1;
#pragma unroll
        for (int i = 0; i < JPT; ++i) {
          const int jo = t + 128 * i;
          if (jo >= NOUT) break;
          const int ox = jo % TXO, oy = jo / TXO;
#pragma unroll
          for (int a = 0; a < 3; ++a)  // z tap a: its three y taps (x already summed), fixed order
            pend[mod3(p2 + 1 - a) * NOUT + jo] +=
                (D3[gofs[i][0] + a * 3 * 128] + D3[gofs[i][1] + a * 3 * 128]) + D3[gofs[i][2] + a * 3 * 128];
          float *pd = pend + mod3(zd) * NOUT + jo;
          const int gx = X0 + ox, gy = Y0 + oy;
          if (zd >= z0 && zd < z1 && gx < NX && gy < NY)
            out[((size_t)zd * NY + gy) * NX + gx] = fmaf(*pd, bias[33], bias[32]);
          *pd = 0.f;
        }
      }
      for (int jo = t; jo < NOUT; jo += 128)  // a new item starts from empty pending planes
        pend[jo] = pend[NOUT + jo] = pend[2 * NOUT + jo] = 0.f;
    }
  }

  fence_before();
  __syncthreads();
  if (warp == 2) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int closure_umma_reserve(ClosureNet *c) {
  if (!c->umw && cudaMalloc(&c->umw, sizeof(UmmaWeights)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  // per device and function; set outside any capture
  if (cudaFuncSetAttribute(closure_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, um::SMEM_B) !=
      cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return 0;
}

cudaError_t closure_umma_prepare(ClosureNet *c, cudaStream_t st) {
  umma_prepare_kernel<<<1, 256, 0, st>>>(c->pb, c->pf, (UmmaWeights *)c->umw);
  return cudaGetLastError();
}

// Work items: output columns of TXO x TYO points times z chunks covering
// the output box; the chunk count minimises the slowest CTA's plane
// iterations, ceil(items / CTAs) x (chunk + 6), the 6 being the z halo of
// the three layers.
cudaError_t closure_umma_run(ClosureNet *c, const void *x16, float *dst, Dims d, const NetBox &box, int *err,
                             cudaStream_t st) {
  if (box.empty()) return cudaSuccess;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 152;
  }
  const int bx = box.hi[0] - box.lo[0], by = box.hi[1] - box.lo[1], bz = box.hi[2] - box.lo[2];
  const int tiles_x = (bx + um::TXO - 1) / um::TXO, tiles_y = (by + um::TYO - 1) / um::TYO;
  const long tiles = (long)tiles_x * tiles_y;
  int best_ch = 1;
  long best_cost = -1;
  const int max_ch = bz / 8 > 1 ? bz / 8 : 1;
  for (int ch = 1; ch <= max_ch; ++ch) {
    const int zc = (bz + ch - 1) / ch;
    const long items = tiles * ((bz + zc - 1) / zc);
    const long cost = ((items + sms - 1) / sms) * (zc + 6);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best_ch = ch;
    }
  }
  const int zc = (bz + best_ch - 1) / best_ch;
  const long nitems = tiles * ((bz + zc - 1) / zc);
  if (nitems > 0x7fffffffL) return cudaErrorInvalidValue;
  const int grid = (int)(nitems < sms ? nitems : sms);
  closure_umma_kernel<<<grid, um::NTHR, um::SMEM_B, st>>>((const uint2 *)x16, (const UmmaWeights *)c->umw, dst,
                                                           d.NX, d.NY, d.NZ, box.lo[0], box.lo[1], box.lo[2],
                                                           box.hi[2], tiles_x, tiles_y, zc, (int)nitems, err);
  return cudaGetLastError();
}

}  // namespace fdw
