// K2: the ct x pt multiply-accumulate of the distance step (Pi_ls step 3,
// f_k = sum_i CMult(c_i, p_ik)).  In the NTT domain CMult is slot-wise, so per
// (query b, block k, component c, prime j, slot s)
//     acc = sum_i ct[b][i][c][j][s] * pt[k][j][i][s]  mod q_j.
//
// The encoded database (d L 8 bytes per point) is streamed from HBM exactly
// once per query; the query ciphertext tile for 64 slots stays in shared
// memory while every block k of that tile streams past it.
//
// Arithmetic: the query values are put in Montgomery form (x 2^64 mod q) and
// both operands are split into 30-bit halves x = x1 2^30 + x0.  The four
// partial products go into four 64-bit accumulators with one 32x32->64
// multiply-add each; 16 products of (2^30 - 1)^2 fit in 64 bits, so every 16
// dimensions the partials are folded into an exact 128-bit sum R.  R < d q^2
// < 2^128 for d <= 224, q < 2^60, and one Montgomery reduction of R gives
// sum_i ct pt mod q below 15 q, finished by four conditional subtractions.
#include "internal.h"

namespace sanns {

namespace {

constexpr int kMacThreads = 512;
constexpr int kMacWarps = kMacThreads / 32;
constexpr uint32_t kSlotTile = 64;  // two slots per lane
constexpr uint32_t kMask30 = (1u << 30) - 1;

struct MacArgs {
  const uint64_t* ct;  // [B][d][2][L][N], NTT form
  const uint64_t* pt;  // [K][L][d][N], NTT form
  uint64_t* out;       // [B][K][2][L][N]
  uint64_t K;
  uint64_t total;      // B L (N / 64) K work items (tile, block)
  uint32_t d;
};

__device__ __forceinline__ void mac4(uint64_t& aL, uint64_t& aM1, uint64_t& aM2, uint64_t& aH,
                                     uint32_t xl, uint32_t xh, uint32_t yl, uint32_t yh) {
  aL += (uint64_t)xl * yl;
  aM1 += (uint64_t)xh * yl;
  aM2 += (uint64_t)xl * yh;
  aH += (uint64_t)xh * yh;
}

__global__ void __launch_bounds__(kMacThreads, 1) mac_kernel(PrimeSet P, MacArgs A) {
  // ct tile: [d][2][32 lanes] x {lo(s0), hi(s0), lo(s1), hi(s1)}
  extern __shared__ uint4 cts[];
  const uint32_t N = P.N, L = P.L, d = A.d;
  const uint32_t tiles = N / kSlotTile;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t w_begin = blockIdx.x * A.total / gridDim.x;
  const uint64_t w_end = (blockIdx.x + 1) * A.total / gridDim.x;

  uint64_t w = w_begin;
  while (w < w_end) {
    const uint64_t u = w / A.K;                     // (b L + j) tiles + st
    const uint64_t k_first = w - u * A.K;
    const uint64_t run_end = min(w_end, (u + 1) * A.K);
    const uint32_t nk = (uint32_t)(run_end - w);
    const uint32_t st = (uint32_t)(u % tiles);
    const uint32_t j = (uint32_t)((u / tiles) % L);
    const uint64_t b = u / ((uint64_t)tiles * L);
    const uint64_t q = P.q[j];

    __syncthreads();  // previous tile fully consumed
    for (uint32_t e = threadIdx.x; e < d * 64; e += kMacThreads) {
      const uint32_t l = e & 31, ci = e >> 5, c = ci & 1, i = ci >> 1;
      const uint64_t* src = A.ct + ((((b * d + i) * 2 + c) * L + j) * N) + st * kSlotTile + 2 * l;
      const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(src);
      const uint64_t m0 = mul_shoup(v.x, P.r64[j], P.r64_shoup[j], q);
      const uint64_t m1 = mul_shoup(v.y, P.r64[j], P.r64_shoup[j], q);
      cts[e] = make_uint4((uint32_t)m0 & kMask30, (uint32_t)(m0 >> 30), (uint32_t)m1 & kMask30,
                          (uint32_t)(m1 >> 30));
    }
    __syncthreads();

    for (uint32_t kk = warp; kk < nk; kk += kMacWarps) {
      const uint64_t k = k_first + kk;
      const uint64_t* p = A.pt + ((k * L + j) * d) * N + st * kSlotTile + 2 * lane;
      u128 R[4];
      uint64_t aL[4], aM1[4], aM2[4], aH[4];
#pragma unroll
      for (int o = 0; o < 4; ++o) { R[o] = 0; aL[o] = aM1[o] = aM2[o] = aH[o] = 0; }

      for (uint32_t i0 = 0; i0 < d; i0 += 16) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          ulonglong2 pv[8];
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const uint32_t i = i0 + 8 * h + v;
            pv[v] = i < d ? __ldcs(reinterpret_cast<const ulonglong2*>(p + (uint64_t)i * N))
                          : make_ulonglong2(0, 0);
          }
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const uint32_t i = i0 + 8 * h + v;
            const uint32_t ii = i < d ? i : d - 1;  // beyond d the pt values are zero
            const uint4 x0 = cts[(ii * 2 + 0) * 32 + lane];
            const uint4 x1 = cts[(ii * 2 + 1) * 32 + lane];
            const uint32_t y0l = (uint32_t)pv[v].x & kMask30, y0h = (uint32_t)(pv[v].x >> 30);
            const uint32_t y1l = (uint32_t)pv[v].y & kMask30, y1h = (uint32_t)(pv[v].y >> 30);
            mac4(aL[0], aM1[0], aM2[0], aH[0], x0.x, x0.y, y0l, y0h);  // c0, slot 0
            mac4(aL[1], aM1[1], aM2[1], aH[1], x0.z, x0.w, y1l, y1h);  // c0, slot 1
            mac4(aL[2], aM1[2], aM2[2], aH[2], x1.x, x1.y, y0l, y0h);  // c1, slot 0
            mac4(aL[3], aM1[3], aM2[3], aH[3], x1.z, x1.w, y1l, y1h);  // c1, slot 1
          }
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const u128 m = (u128)aM1[o] + aM2[o];
          R[o] += (u128)aL[o] + (m << 30) + ((u128)aH[o] << 60);
          aL[o] = aM1[o] = aM2[o] = aH[o] = 0;
        }
      }
      const uint64_t qn = P.q_neg_inv[j];
      uint64_t r[4];
#pragma unroll
      for (int o = 0; o < 4; ++o) r[o] = reduce_below_16q(redc128(R[o], q, qn), q);
      uint64_t* o0 = A.out + (((b * A.K + k) * 2 + 0) * L + j) * N + st * kSlotTile + 2 * lane;
      uint64_t* o1 = A.out + (((b * A.K + k) * 2 + 1) * L + j) * N + st * kSlotTile + 2 * lane;
      *reinterpret_cast<ulonglong2*>(o0) = make_ulonglong2(r[0], r[1]);
      *reinterpret_cast<ulonglong2*>(o1) = make_ulonglong2(r[2], r[3]);
    }
    w = run_end;
  }
}

}  // namespace

cudaError_t launch_mac(const PrimeSet& P, const uint64_t* ct, const uint64_t* pt, uint32_t B,
                       uint32_t d, uint64_t K, uint64_t* out, int sms, cudaStream_t st) {
  MacArgs A;
  A.ct = ct;
  A.pt = pt;
  A.out = out;
  A.K = K;
  A.d = d;
  A.total = (uint64_t)B * P.L * (P.N / kSlotTile) * K;
  if (A.total == 0) return cudaSuccess;
  const size_t smem = sizeof(uint4) * 64 * d;
  cudaError_t e = cudaFuncSetAttribute(mac_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  uint64_t grid = (uint64_t)(sms > 0 ? sms : 148);
  if (grid > A.total) grid = A.total;
  mac_kernel<<<(unsigned)grid, kMacThreads, smem, st>>>(P, A);
  return cudaGetLastError();
}

}  // namespace sanns
