// closure_tc.cu -- inference of the learned closure on the tensor cores.
//
// The network (closure.cu: three 3x3x3 convolutions 3 -> 16 -> 16 -> 1,
// ReLU between, zero padding at every layer) is evaluated on a whole
// computational grid by one kernel that marches z planes and keeps every
// intermediate activation on chip:
//   input ring  : 3 planes of x = (u/s, u_{n-1}/s, v', 0) in FP16,
//   layer-1 ring: 3 planes of a1 (16 channels, FP16),
//   layer 2     : the current plane of a2 (FP16),
//   layer 3     : per-tap products of the current a2 plane (FP32), gathered
//                 into three pending output planes (FP32).
// Two barriers per plane: [layer-3 gather of the previous plane + layer 1]
// | [layer 2 and the layer-3 products of each warp's own layer-2 tile + the
// next input plane (prefetched into registers one plane ahead)].
// Layers 1 and 2 are implicit GEMMs on mma.sync.m16n8k16 (FP16 operands,
// FP32 accumulation) with the weights as the 16 x 16 A operand (rows =
// output channels) and 8 points along x as B; one B fragment serves the
// three taps that differ in y. Layer 3 has one output channel, so its GEMM
// runs the other way round: M = the 27 taps (32), N = 8 points, K = 16
// channels, and the 27 products of a point are summed by a gather. The
// weights are the BF16 parameters converted exactly to FP16 (the last layer
// scaled by a power of two into FP16's normal range and scaled back in
// FP32). Every reduction has a fixed order: the kernel is deterministic, so
// net(x0) computed once and net(x) agree bit for bit where the wavefield is
// zero.
#include <math.h>
#include <stdint.h>

#include "fdw_internal.h"
#include "fdwave.h"

namespace fdw {

namespace tc {

constexpr int TX = 30, TY = 14;      // output tile of a CTA (per plane)
constexpr int W2R = 32, H2R = 16;    // layer-2 region (TX + 2, TY + 2)
constexpr int W1R = 40, H1R = 18;    // layer-1 region computed (TX + 4 = 34 needed; 5 x 8 columns)
constexpr int WI = 44, HI = 20;      // input region (W1R + 4 for the 4-point K window, H1R + 2)
constexpr int WIS = 46;              // row length (points) of both input copies
// The odd-shifted copy starts 48 bytes (mod 128) after the even one, so that
// the 16-byte rows of one ldmatrix phase (8 consecutive points: 4 from each
// copy) fall on disjoint bank groups.
constexpr int IN_E_B = HI * WIS * 8 + 112;     // one input plane, even copy (+ bank offset)
constexpr int NWARP = 16, NTHR = 32 * NWARP;
constexpr int DSTR = W2R * H2R + 8;  // row stride (floats) of the layer-3 product buffer

// shared memory layout (bytes)
constexpr int IN_O_B = HI * WIS * 8;           // one input plane, odd-shifted copy
constexpr int IN_PLANE_B = IN_E_B + IN_O_B;
constexpr int A1_PLANE_B = H1R * W1R * 32;     // 16 FP16 channels per point
constexpr int A2_B = H2R * W2R * 32;
constexpr int D3_B = 32 * DSTR * 4;
constexpr int O_PLANE_B = TY * TX * 4;
constexpr int W1_B = 9 * 256 * 2;              // [a*3+b][co][k]
constexpr int W2_B = 27 * 256 * 2;             // [tap][co][ci]
constexpr int W3_B = 32 * 16 * 2;              // [tap][ci]
constexpr int OFF_IN = 0;
constexpr int OFF_A1 = OFF_IN + 3 * IN_PLANE_B;
constexpr int OFF_A2 = OFF_A1 + 3 * A1_PLANE_B;
constexpr int OFF_D3 = OFF_A2 + A2_B;
constexpr int OFF_O = OFF_D3 + D3_B;
constexpr int OFF_W1 = OFF_O + 3 * O_PLANE_B;
constexpr int OFF_W2 = OFF_W1 + W1_B;
constexpr int OFF_W3 = OFF_W2 + W2_B;
constexpr int OFF_B = OFF_W3 + W3_B;           // b1[16], b2[16], b3, 2^-e3 (floats)
constexpr int SMEM_B = OFF_B + 64 * 4;
static_assert(SMEM_B <= 227 * 1024, "shared memory per CTA");
static_assert(IN_E_B % 128 == 48 && IN_PLANE_B % 16 == 0 && A1_PLANE_B % 16 == 0 && A2_B % 16 == 0 &&
                  OFF_W1 % 16 == 0 && OFF_W2 % 16 == 0 && OFF_W3 % 16 == 0,
              "16-byte alignment of ldmatrix rows");

}  // namespace tc

// Weights of the tensor-core kernel, prepared on the device from the
// closure's parameters (pb: BF16 copies, pf: FP32 masters).
struct TcWeights {
  __half w1[9 * 256];   // [a*3+b][co][k = 4 cx + ci], cx = x offset + 1 (3: zero), ci < 3
  __half w2[27 * 256];  // [tap][co][ci]
  __half w3[32 * 16];   // [tap][ci] times 2^e3, taps >= 27 zero
  float b1[16], b2[16], b3, w3_unscale;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                        uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t &r0, uint32_t &r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}
// D += A (16x16, FP16) * B (16x8, FP16), FP32 accumulators. Not volatile:
// it only reads and writes registers, so the compiler may schedule it
// after later (volatile) fragment loads and hide their latency.
__device__ __forceinline__ void mma16816(float *d, const uint32_t *a, uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t s_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of channel half h (0: channels 0-7, 1: 8-15) of point q in a
// 16-channel activation row; the halves are swapped for points with bit 2
// set so that 8 consecutive points of an ldmatrix phase hit 8 bank groups.
__device__ __forceinline__ int act_off(int q, int h) { return q * 32 + ((h ^ ((q >> 2) & 1)) << 4); }

// Epilogue of a 16 (channels) x 8 (points) FP32 accumulator tile: bias,
// ReLU, zero for points outside the grid, FP16, stored as the 16-channel
// rows of points q0 .. q0+7 (act_off layout). The lane holds channels g and
// g+8 of points 2t, 2t+1 -- rows of the two 8 x 8 [channel][point] halves;
// stmatrix .trans writes their transposes, one point per row.
__device__ __forceinline__ void store_act_tile(unsigned char *base, int q0, const float *acc, float blo,
                                               float bhi, bool in0, bool in1, int lane) {
  const float v00 = in0 ? fmaxf(acc[0] + blo, 0.f) : 0.f, v01 = in1 ? fmaxf(acc[1] + blo, 0.f) : 0.f;
  const float v10 = in0 ? fmaxf(acc[2] + bhi, 0.f) : 0.f, v11 = in1 ? fmaxf(acc[3] + bhi, 0.f) : 0.f;
  __half2 h0 = __floats2half2_rn(v00, v01), h1 = __floats2half2_rn(v10, v11);
  const uint32_t r0 = *reinterpret_cast<uint32_t *>(&h0), r1 = *reinterpret_cast<uint32_t *>(&h1);
  const uint32_t addr = s_u32(base + act_off(q0 + (lane & 7), (lane >> 3) & 1));
  asm volatile("stmatrix.sync.aligned.m8n8.x2.trans.shared.b16 [%0], {%1, %2};" ::"r"(addr), "r"(r0), "r"(r1)
               : "memory");
}

// A fragment (16 x 16, row-major [m][k] FP16 in shared memory, each row's
// 16-byte halves placed by act_off) of ldmatrix.x4.
__device__ __forceinline__ void load_a(const __half *m, int lane, uint32_t *a) {
  const int r = (lane & 7) + ((lane >> 3) & 1) * 8, h = lane >> 4;
  ldsm_x4(s_u32(reinterpret_cast<const unsigned char *>(m) + act_off(r, h)), a[0], a[1], a[2], a[3]);
}

// ---------------------------------------------------------------------------
// weight preparation (one block)
// ---------------------------------------------------------------------------
__global__ void tc_prepare_kernel(const __nv_bfloat16 *__restrict__ pb, const float *__restrict__ pf,
                                  TcWeights *__restrict__ w) {
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
  // 2^e3 max|W3| in [1, 2): exact scaling into FP16's normal range
  const int e3 = amax[0] > 0.f ? -ilogbf(amax[0]) : 0;
  for (int i = t; i < 9 * 256; i += blockDim.x) {
    const int ab = i / 256, co = (i / 16) % 16, k = i % 16, cx = k / 4, ci = k % 4;
    float v = 0.f;
    if (cx < 3 && ci < 3) v = __bfloat162float(pb[OW1 + (co * 3 + ci) * 27 + ab * 3 + cx]);
    w->w1[i] = __float2half_rn(v);
  }
  for (int i = t; i < 27 * 256; i += blockDim.x) {
    const int tap = i / 256, co = (i / 16) % 16, ci = i % 16;
    w->w2[i] = __float2half_rn(__bfloat162float(pb[OW2 + (co * H + ci) * 27 + tap]));
  }
  for (int i = t; i < 32 * 16; i += blockDim.x) {
    const int tap = i / 16, ci = i % 16;
    const float v = tap < 27 ? ldexpf(__bfloat162float(pb[OW3 + ci * 27 + tap]), e3) : 0.f;
    w->w3[i] = __float2half_rn(v);
  }
  if (t < 16) {
    w->b1[t] = pf[OB1 + t];
    w->b2[t] = pf[OB2 + t];
  }
  if (t == 0) {
    w->b3 = pf[OB3];
    w->w3_unscale = ldexpf(1.f, -e3);
  }
}

// x16[p] = (u/s, u_{n-1}/s, (v - 3000)/750, 0) in FP16, dense [NZ][NY][NX];
// u == null gives the zero-wavefield input x0.
template <typename T>
__global__ void tc_inputs_kernel(const T *__restrict__ u, const T *__restrict__ um,
                                 const float *__restrict__ vp, int nx, int ny, int nz, int nb, Dims d,
                                 const float *__restrict__ s_dev, uint2 *__restrict__ x16) {
  const float inv = u ? 1.f / *s_dev : 0.f;
  const int rows = d.NY * d.NZ;  // one block per row: no 64-bit division per point
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % d.NY, k = row / d.NY;
    const float *vr = vp + ((size_t)min(max(k - nb, 0), nz - 1) * ny + min(max(j - nb, 0), ny - 1)) * nx;
    for (int i = threadIdx.x; i < d.NX; i += blockDim.x) {
      const size_t p = (size_t)row * d.Xp + i;
      const float v = (vr[min(max(i - nb, 0), nx - 1)] - 3000.f) / 750.f;
      const float a = u ? St<T>::ld(u[p]) * inv : 0.f, b = u ? St<T>::ld(um[p]) * inv : 0.f;
      __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(v, 0.f);
      uint2 o;
      o.x = *reinterpret_cast<uint32_t *>(&lo);
      o.y = *reinterpret_cast<uint32_t *>(&hi);
      x16[(size_t)row * d.NX + i] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// the fused network kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(tc::NTHR, 1)
    closure_tc_kernel(const uint2 *__restrict__ x16, const TcWeights *__restrict__ wg, float *__restrict__ out,
                      int NX, int NY, int NZ, int ox, int oy, int oz, int zend, int zc) {
  using namespace tc;
  extern __shared__ __align__(16) unsigned char sm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int X0 = ox + blockIdx.x * TX, Y0 = oy + blockIdx.y * TY;
  const int z0 = oz + blockIdx.z * zc, z1 = min(z0 + zc, zend);
  if (z0 >= z1) return;

  // weights and biases into shared memory; each 16 x 16 matrix's rows are
  // laid out by act_off (row r's halves swapped when bit 2 of r is set)
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(wg->w1);
    constexpr int n16 = (W1_B + W2_B + W3_B) / 16;  // w1 | w2 | w3 are contiguous in TcWeights
    for (int i = tid; i < n16; i += NTHR) {
      const int mat = i >> 5, r = (i >> 1) & 15, h = i & 1;  // 32 16-byte pieces per matrix
      *reinterpret_cast<uint4 *>(sm + OFF_W1 + mat * 512 + act_off(r, h)) = src[i];
    }
    float *bsm = reinterpret_cast<float *>(sm + OFF_B);
    if (tid < 16) {
      bsm[tid] = wg->b1[tid];
      bsm[16 + tid] = wg->b2[tid];
    }
    if (tid == 0) {
      bsm[32] = wg->b3;
      bsm[33] = wg->w3_unscale;
    }
    float *o = reinterpret_cast<float *>(sm + OFF_O);
    for (int i = tid; i < 3 * TY * TX; i += NTHR) o[i] = 0.f;
  }
  __syncthreads();
  const __half *W1s = reinterpret_cast<const __half *>(sm + OFF_W1);
  const __half *W2s = reinterpret_cast<const __half *>(sm + OFF_W2);
  const __half *W3s = reinterpret_cast<const __half *>(sm + OFF_W3);
  const float *bsm = reinterpret_cast<const float *>(sm + OFF_B);


  const int g = lane >> 2, t4 = lane & 3;  // fragment row group / column pair
  // output planes [z0, z1) need a2 planes z0-1 .. z1, a1 planes z0-2 .. z1+1
  // and input planes z0-3 .. z1+2: one input plane per iteration
  const int nit = (z1 - z0) + 6;

  // Input planes go global -> registers one iteration ahead, registers ->
  // ring slot at the end of the previous iteration: the global latency
  // overlaps the MMA phases.
  constexpr int NPF = (HI * WI + NTHR - 1) / NTHR;
  uint2 pf[NPF];
  auto fetch = [&](int zi) {
    const bool zin = zi >= 0 && zi < NZ;
#pragma unroll
    for (int k = 0; k < NPF; ++k) {
      const int i = tid + k * NTHR;
      const int yi = i / WI, xi = i % WI;
      const int y = Y0 - 3 + yi, x = X0 - 3 + xi;
      pf[k] = make_uint2(0u, 0u);
      if (i < HI * WI && zin && y >= 0 && y < NY && x >= 0 && x < NX) pf[k] = x16[((size_t)zi * NY + y) * NX + x];
    }
  };
  auto store = [&](int zi) {
    const int slot = ((zi % 3) + 3) % 3;
    uint2 *E = reinterpret_cast<uint2 *>(sm + OFF_IN + slot * IN_PLANE_B);
    uint2 *O = reinterpret_cast<uint2 *>(sm + OFF_IN + slot * IN_PLANE_B + IN_E_B);
#pragma unroll
    for (int k = 0; k < NPF; ++k) {
      const int i = tid + k * NTHR;
      if (i < HI * WI) {
        const int yi = i / WI, xi = i % WI;
        E[yi * WIS + xi] = pf[k];
        O[yi * WIS + xi + 1] = pf[k];
      }
    }
    if (tid < HI) {  // odd copy: slots 0 and WIS-1 are never read as data; keep them finite
      O[tid * WIS] = make_uint2(0u, 0u);
      O[tid * WIS + WIS - 1] = make_uint2(0u, 0u);
    }
  };
  fetch(z0 - 3);
  store(z0 - 3);
  fetch(z0 - 2);
  __syncthreads();

  // Layer-3 gather of a2 plane p's products (D) into the pending output
  // planes p+1 (a = 0), p (a = 1), p-1 (a = 2); plane p-1 is then complete
  // and written out. Runs one iteration after the products, together with
  // the next plane's layer 1 (two barriers per plane).
  auto gather = [&](int p) {
    const float *D = reinterpret_cast<const float *>(sm + OFF_D3);
    float *O = reinterpret_cast<float *>(sm + OFF_O);
    for (int i = tid; i < TY * TX; i += NTHR) {
      const int oy = i / TX, ox = i % TX;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int zo = p + 1 - a;
        float sacc = 0.f;
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int c = 0; c < 3; ++c) sacc += D[((a * 3 + b) * 3 + c) * DSTR + (oy + b) * W2R + ox + c];
        O[(((zo % 3) + 3) % 3) * TY * TX + i] += sacc;
      }
      const int zd = p - 1;  // complete
      float *Od = O + (((zd % 3) + 3) % 3) * TY * TX + i;
      const int gy = Y0 + oy, gx = X0 + ox;
      if (zd >= z0 && zd < z1 && gy < NY && gx < NX)
        out[((size_t)zd * NY + gy) * NX + gx] = fmaf(*Od, bsm[33], bsm[32]);
      *Od = 0.f;  // the slot is reused for plane p + 2
    }
  };

  for (int j = 0; j < nit; ++j) {
    const int zi = z0 - 3 + j;  // the newest input plane in the ring
    if (j >= 5) gather(zi - 3);  // products of the previous iteration's layer-2 plane
    // ---- P1: layer 1 at plane q1 = zi - 1 (input planes q1-1 .. q1+1)
    const int q1 = zi - 1;
    if (j >= 2) {
      unsigned char *a1p = sm + OFF_A1 + (((q1 % 3) + 3) % 3) * A1_PLANE_B;
      const bool zin = q1 >= 0 && q1 < NZ;
      constexpr int RY = 6, NSTRIP = W1R / 8, NBLK = H1R / RY;  // 5 x 3 items
      for (int item = warp; item < NSTRIP * NBLK; item += NWARP) {
        const int sx = item % NSTRIP, yb = (item / NSTRIP) * RY;
        float acc[RY][4];
#pragma unroll
        for (int r = 0; r < RY; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
        // B rows: lanes 0-7 point n = lane (k 0-7 = points x-1, x), lanes
        // 8-15 the same points (k 8-15 = points x+1, x+2)
        const int n = lane & 7, hk = (lane >> 3) & 1;
        const int x1 = sx * 8 + n;          // layer-1 region column of the point
        const int xi = x1 + 2 * hk;         // first input column of the 16-byte row
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int pz = q1 + a - 1;
          const unsigned char *inp = sm + OFF_IN + (((pz % 3) + 3) % 3) * IN_PLANE_B;
          uint32_t aw[3][4];
#pragma unroll
          for (int b = 0; b < 3; ++b) load_a(W1s + (a * 3 + b) * 256, lane, aw[b]);
          // row yi of the input plane as this lane's ldmatrix row address
          auto row_addr = [&](int yi) {
            return (xi & 1) ? s_u32(inp + IN_E_B + (yi * WIS + xi + 1) * 8) : s_u32(inp + (yi * WIS + xi) * 8);
          };
          uint32_t bc0, bc1;
          ldsm_x2(row_addr(yb), bc0, bc1);
#pragma unroll
          for (int yy = 0; yy < RY + 2; ++yy) {  // input row yb + yy = layer-1 row + b
            uint32_t bn0 = 0u, bn1 = 0u;
            if (yy + 1 < RY + 2) ldsm_x2(row_addr(yb + yy + 1), bn0, bn1);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
              const int r = yy - b;
              if (r >= 0 && r < RY) mma16816(acc[r], aw[b], bc0, bc1);
            }
            bc0 = bn0;
            bc1 = bn1;
          }
        }
        // epilogue: bias, ReLU, zero outside the grid, FP16 into the ring
        const int gx0 = X0 - 2 + sx * 8 + 2 * t4;
        const bool xin0 = gx0 >= 0 && gx0 < NX, xin1 = gx0 + 1 >= 0 && gx0 + 1 < NX;
        const float blo = bsm[g], bhi = bsm[g + 8];
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int y1 = yb + r, gy = Y0 - 2 + y1;
          const bool yin = zin && gy >= 0 && gy < NY;
          store_act_tile(a1p, y1 * W1R + sx * 8, acc[r], blo, bhi, yin && xin0, yin && xin1, lane);
        }
      }
    }
    __syncthreads();

    // ---- P2: layer 2 at plane q2 = zi - 2 (layer-1 planes q2-1 .. q2+1)
    const int q2 = zi - 2;
    if (j >= 4) {
      const bool zin = q2 >= 0 && q2 < NZ;
      unsigned char *a2p = sm + OFF_A2;
      constexpr int RY = 4, NSTRIP = W2R / 8, NBLK = H2R / RY;  // 4 x 4 items
      for (int item = warp; item < NSTRIP * NBLK; item += NWARP) {
        const int sx = item % NSTRIP, yb = (item / NSTRIP) * RY;
        float acc[RY][4];
#pragma unroll
        for (int r = 0; r < RY; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
        const int n = lane & 7, hk = (lane >> 3) & 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int pz = q2 + a - 1;
          const unsigned char *a1p = sm + OFF_A1 + (((pz % 3) + 3) % 3) * A1_PLANE_B;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            uint32_t aw[3][4];
#pragma unroll
            for (int b = 0; b < 3; ++b) load_a(W2s + ((a * 3 + b) * 3 + c) * 256, lane, aw[b]);
            const int x1 = sx * 8 + n + c;  // layer-1 column = layer-2 column + c
            // B fragments one row ahead of the MMAs that use them
            uint32_t bc0, bc1;
            ldsm_x2(s_u32(a1p + act_off(yb * W1R + x1, hk)), bc0, bc1);
#pragma unroll
            for (int yy = 0; yy < RY + 2; ++yy) {
              uint32_t bn0 = 0u, bn1 = 0u;
              if (yy + 1 < RY + 2) ldsm_x2(s_u32(a1p + act_off((yb + yy + 1) * W1R + x1, hk)), bn0, bn1);
#pragma unroll
              for (int b = 0; b < 3; ++b) {
                const int r = yy - b;  // layer-1 row yb + yy = layer-2 row yb + r, plus b
                if (r >= 0 && r < RY) mma16816(acc[r], aw[b], bc0, bc1);
              }
              bc0 = bn0;
              bc1 = bn1;
            }
          }
        }
        {
          const int gx0 = X0 - 1 + sx * 8 + 2 * t4;
          const bool xin0 = gx0 >= 0 && gx0 < NX, xin1 = gx0 + 1 >= 0 && gx0 + 1 < NX;
          const float blo = bsm[16 + g], bhi = bsm[16 + g + 8];
#pragma unroll
          for (int r = 0; r < RY; ++r) {
            const int y2 = yb + r, gy = Y0 - 1 + y2;
            const bool yin = zin && gy >= 0 && gy < NY;
            store_act_tile(a2p, y2 * W2R + sx * 8, acc[r], blo, bhi, yin && xin0, yin && xin1, lane);
          }
        }
        // layer-3 products of this warp's own a2 points (the rows of the
        // item are whole 8-point n-tiles): D[tap][point] = sum_ci W3 a2
        __syncwarp();
        float *D = reinterpret_cast<float *>(sm + OFF_D3);
        uint32_t a3w[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) load_a(W3s + mt * 256, lane, a3w[mt]);
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          const int nt = (yb + r) * (W2R / 8) + sx;
          uint32_t b0, b1;
          ldsm_x2(s_u32(a2p + act_off(nt * 8 + n, hk)), b0, b1);
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            float d3[4] = {0.f, 0.f, 0.f, 0.f};
            mma16816(d3, a3w[mt], b0, b1);
            const int tap = mt * 16 + g, pt = nt * 8 + 2 * t4;
            *reinterpret_cast<float2 *>(D + tap * DSTR + pt) = make_float2(d3[0], d3[1]);
            *reinterpret_cast<float2 *>(D + (tap + 8) * DSTR + pt) = make_float2(d3[2], d3[3]);
          }
        }
        __syncwarp();  // the a2 tile is rewritten by this warp in the next plane
      }
    }
    // next input plane into the slot of plane zi - 2 (last read by layer 1
    // of this iteration, one barrier ago), then prefetch the one after
    if (j + 1 < nit) {
      store(zi + 1);
      if (j + 2 < nit) fetch(zi + 2);
    }
    __syncthreads();

  }
  if (nit - 1 >= 4) gather(z0 - 3 + nit - 1 - 2);  // products of the last layer-2 plane
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int closure_tc_reserve(ClosureNet *c, Dims d) {
  const size_t vol = (size_t)d.NX * d.NY * d.NZ;
  if (c->variant == 0 && closure_umma_reserve(c)) return -1;
  if (c->tc_cap >= vol && c->tcw) return 0;
  cudaFree(c->x16);
  cudaFree(c->tc_out);
  c->x16 = nullptr;
  c->tc_out = nullptr;
  c->tc_cap = 0;
  if (cudaMalloc(&c->x16, vol * 8) != cudaSuccess || cudaMalloc(&c->tc_out, vol * 4) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (!c->tcw && cudaMalloc(&c->tcw, sizeof(TcWeights)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  c->tc_cap = vol;
  // per device and function; set on every (re)allocation, outside any capture
  if (cudaFuncSetAttribute(closure_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_B) !=
      cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return 0;
}

// net(x) into `dst` (FP32 dense [NZ][NY][NX]) on the output box, the
// points the correction is applied to; u == null: x0. Variant 0 runs the
// tcgen05 kernel, variant 2 the mma.sync kernel.
template <typename T>
static cudaError_t tc_net(ClosureNet *c, const T *u, const T *um, const float *vp, int nx, int ny, int nz, int nb,
                          Dims d, float *dst, int *err, cudaStream_t st) {
  const long rows = (long)d.NY * d.NZ;
  tc_inputs_kernel<T><<<(int)(rows < 152 * 64 ? rows : 152 * 64), 256, 0, st>>>(u, um, vp, nx, ny, nz, nb, d,
                                                                                c->s_dev, (uint2 *)c->x16);
  const int n[3] = {nx, ny, nz};
  NetBox box;
  for (int a = 0; a < 3; ++a) {
    box.lo[a] = nb + kClosureHalo;
    box.hi[a] = nb + n[a] - kClosureHalo;
  }
  if (c->variant == 0) return closure_umma_run(c, c->x16, dst, d, box, err, st);
  if (box.empty()) return cudaGetLastError();
  const int bx = box.hi[0] - box.lo[0], by = box.hi[1] - box.lo[1], bz = box.hi[2] - box.lo[2];
  const int tiles = ((bx + tc::TX - 1) / tc::TX) * ((by + tc::TY - 1) / tc::TY);
  int zch = (2 * 152 + tiles - 1) / tiles;  // about two CTAs per SM in total
  if (zch < 1) zch = 1;
  const int zmax = bz / 16 > 0 ? bz / 16 : 1;  // chunks of >= 16 planes (the z halo is 5 planes)
  if (zch > zmax) zch = zmax;
  const int zc = (bz + zch - 1) / zch;
  dim3 grd((bx + tc::TX - 1) / tc::TX, (by + tc::TY - 1) / tc::TY, (bz + zc - 1) / zc);
  closure_tc_kernel<<<grd, tc::NTHR, tc::SMEM_B, st>>>((const uint2 *)c->x16, (const TcWeights *)c->tcw, dst,
                                                       d.NX, d.NY, d.NZ, box.lo[0], box.lo[1], box.lo[2],
                                                       box.hi[2], zc);
  return cudaGetLastError();
}

cudaError_t closure_tc_base(ClosureNet *c, const float *vp, int nx, int ny, int nz, int nb, Dims d, int *err,
                            cudaStream_t st) {
  cudaError_t e;
  if (c->variant == 0) {
    e = closure_umma_prepare(c, st);
  } else {
    tc_prepare_kernel<<<1, 256, 0, st>>>(c->pb, c->pf, (TcWeights *)c->tcw);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  return tc_net<float>(c, nullptr, nullptr, vp, nx, ny, nz, nb, d, c->base, err, st);
}

cudaError_t closure_tc_net(ClosureNet *c, int storage, const void *u, const void *um, const float *vp, int nx,
                           int ny, int nz, int nb, Dims d, int *err, cudaStream_t st) {
  switch (storage) {
    case FDW_F32:
      return tc_net<float>(c, (const float *)u, (const float *)um, vp, nx, ny, nz, nb, d, c->tc_out, err, st);
    case FDW_BF16:
      return tc_net<__nv_bfloat16>(c, (const __nv_bfloat16 *)u, (const __nv_bfloat16 *)um, vp, nx, ny, nz, nb, d,
                                   c->tc_out, err, st);
    case FDW_F16:
      return tc_net<__half>(c, (const __half *)u, (const __half *)um, vp, nx, ny, nz, nb, d, c->tc_out, err, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fdw
