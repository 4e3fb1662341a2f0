// K5: the batched ct x pt MAC on the tensor cores (tcgen05, kind::f16, bf16
// operands, fp32 accumulation in TMEM), exact.
//
// With B queries, every (prime j, slot s) is the contraction
//     C[(b, c)][k] = sum_i A[(b, c)][i] P[k][i]  mod q_j,
// A = the query ciphertexts (NTT form), P = the encoded database.  Residues
// are split into balanced base-256 digits in [-128, 127], which bf16 holds
// exactly.  The database side is split once, P[k][i] = sum_b p_b 256^b; the
// query side is folded with the digit weight of the database side,
// X_b = A 256^b mod q = sum_a x_{b,a} 256^a, so that
//     C = sum_a 256^a S_a,   S_a = sum_{i, b} x_{b,a}[i] p_b[k][i]   (mod q).
// S_a is one GEMM with rows (b, c, a), columns k and contraction (i, b):
// every product is at most 2^14 in magnitude and a sum of 8 d <= 1024 of them
// stays within 2^24, so the fp32 accumulation is exact for d <= 128.
//
// One persistent CTA per SM, warp-specialised:
//   warp 0      TMA producer: database digit tile (256 rows x 64 bf16) per stage
//   warp 1      TMEM owner and MMA issuer (one thread): 4 MMAs of
//               M = 128, N = 256, K = 16 per stage
//   warps 2-5   query-digit producers: 128 rows x 64 bf16 per stage, written
//               into shared memory in the 128-byte swizzled layout
//   warps 6-13  epilogue: TMEM -> registers -> int32, transposed through
//               shared memory so each lane combines the 8 digit rows of one
//               output exactly, store acc[b][k][c][j][s]
// Work unit = (prime, slot, 256-column N tile, 16-row M tile), M tile fastest,
// so the CTAs running side by side share each database tile through L2.
// Every wait is bounded: on time-out the kernel raises a device error flag,
// drains its own copies, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "internal.h"

namespace sanns {

namespace {

constexpr int kStages = 4;
constexpr int kBM = 128;                 // rows (b, c, a) per tile: 16 (b, c) x 8 digits
constexpr int kBN = 256;                 // database blocks per tile
constexpr int kBK = 64;                  // contraction columns (8 dims x 8 digits) per stage
constexpr int kATile = kBM * kBK * 2;    // 16 KB
constexpr int kBTile = kBN * kBK * 2;    // 32 KB
constexpr int kStageBytes = kATile + kBTile;
constexpr int kProdWarp0 = 2;
constexpr int kProdWarps = 4;
constexpr int kProdThreads = 32 * kProdWarps;
static_assert(kProdThreads == 16 * 8, "one (row group, dimension) item per producer thread");
constexpr int kEpiWarp0 = kProdWarp0 + kProdWarps;   // 6
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (kEpiWarp0 + kEpiWarps);  // 448
constexpr int kEpiCols = 16;                             // TMEM columns per load
constexpr int kTrStride = kEpiCols + 1;                  // padded transpose row (words)
constexpr unsigned long long kWaitCycles = 4ull << 30;  // ~2 s at 2 GHz

struct BatchArgs {
  const uint64_t* ct;     // [B][d][2][L][N]
  uint64_t* out;          // [B][K][2][L][N]
  int* err;               // device error word
  uint32_t B, d, dpad, K;
  uint32_t MT, NT, chunks;
  uint64_t units;
  uint64_t w256[kMaxPrimes][8];        // 256^a mod q_j
  uint64_t w256_shoup[kMaxPrimes][8];
  uint64_t r256_shoup[kMaxPrimes];     // Shoup companion of 256
  uint64_t w32[kMaxPrimes];            // 2^32 mod q_j
  uint64_t w32_shoup[kMaxPrimes];
  uint64_t mu64[kMaxPrimes];           // floor(2^64 / q_j)
};

// |v| mod q for |v| < 2^63 with mu = floor(2^64 / q), returned as v mod q.
__device__ __forceinline__ uint64_t signed_mod(int64_t v, uint64_t q, uint64_t mu) {
  const uint64_t m = v >= 0 ? (uint64_t)v : (uint64_t)(-v);
  const uint64_t r = mod_t64(m, q, mu);
  return (v >= 0 || r == 0) ? r : q - r;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false when the CTA is aborting or the wait timed out (which
// also raises the abort flag and the device error word).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, uint32_t sleep_ns = 0) {
  const unsigned long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (sleep_ns && it > 2) __nanosleep(sleep_ns);
    if ((it & 255) == 255) {
      if (*abort_flag) return false;
      if (clock64() - t0 > kWaitCycles) {
        *abort_flag = 1;
        atomicExch(err, SANNS_ETIMEOUT);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// K-major operand, 128-byte rows, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// kind::f16: D fp32, A and B bf16, both K-major, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

struct Decoded {
  uint32_t j, mt, nt, s;
};

// unit = ((j N + s) NT + nt) MT + mt: the M tiles of one database tile are
// consecutive, so CTAs running side by side share it through L2.
__device__ __forceinline__ Decoded decode_unit(uint64_t u, uint32_t N, const BatchArgs& A) {
  Decoded D;
  D.mt = (uint32_t)(u % A.MT);
  uint64_t r = u / A.MT;
  D.nt = (uint32_t)(r % A.NT);
  r /= A.NT;
  D.s = (uint32_t)(r % N);
  D.j = (uint32_t)(r / N);
  return D;
}

__global__ void __launch_bounds__(kThreads, 1)
batched_mac_kernel(const __grid_constant__ CUtensorMap pmap, PrimeSet P, BatchArgs A) {
  extern __shared__ __align__(1024) uint8_t dsmem[];
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages];
  __shared__ __align__(8) uint64_t bar_tfull[2], bar_tempty[2];
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;
  __shared__ int32_t tr[kEpiWarps][32 * kTrStride];

  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* base = dsmem + ((1024 - (smem_u32(dsmem) & 1023)) & 1023);
  const uint32_t sbase = smem_u32(base);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 2);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bar_tfull[a]), 1);
      mbar_init(smem_u32(&bar_tempty[a]), kEpiWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&tmem_base_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;
  const uint32_t N = P.N, L = P.L;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint64_t g = 0;
      for (uint64_t u = blockIdx.x; u < A.units && !abort_flag; u += gridDim.x) {
        const Decoded D = decode_unit(u, N, A);
        for (uint32_t kc = 0; kc < A.chunks; ++kc, ++g) {
          const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
          if (!mbar_wait(smem_u32(&bar_empty[st]), ph ^ 1, &abort_flag, A.err)) break;
          const uint32_t full = smem_u32(&bar_full[st]);
          mbar_arrive_tx(full, kBTile);
          tma_load_3d(sbase + st * kStageBytes + kATile, &pmap, (int)(kc * kBK), (int)(D.nt * kBN),
                      (int)(D.j * N + D.s), full);
        }
      }
      // drain: every issued copy completes before the CTA may exit
      if (abort_flag) {
        const uint64_t first = g > kStages ? g - kStages : 0;
        for (uint64_t h = first; h < g; ++h) {
          const uint32_t st = (uint32_t)(h % kStages), ph = (uint32_t)((h / kStages) & 1);
          const unsigned long long t0 = clock64();
          while (!mbar_try(smem_u32(&bar_full[st]), ph) && clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint64_t g = 0, r = 0;
      for (uint64_t u = blockIdx.x; u < A.units && !abort_flag; u += gridDim.x, ++r) {
        const uint32_t slot = (uint32_t)(r & 1), aph = (uint32_t)((r >> 1) & 1);
        if (!mbar_wait(smem_u32(&bar_tempty[slot]), aph ^ 1, &abort_flag, A.err)) break;
        tc_fence_after();
        const uint32_t dt = tmem + slot * kBN;
        bool ok = true;
        for (uint32_t kc = 0; kc < A.chunks; ++kc, ++g) {
          const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
          if (!mbar_wait(smem_u32(&bar_full[st]), ph, &abort_flag, A.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a_addr = sbase + st * kStageBytes, b_addr = a_addr + kATile;
          const uint64_t ad = smem_desc(a_addr), bd = smem_desc(b_addr);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k)
            mma_bf16(dt, ad + 2 * k, bd + 2 * k, (kc > 0 || k > 0) ? 1u : 0u);
          mma_commit(smem_u32(&bar_empty[st]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&bar_tfull[slot]));
      }
    }
  } else if (warp < kEpiWarp0) {
    // ---------------- query-digit producers ----------------
    // Balanced base-256 digits of X in [-128, 127]: the bytes of
    // X + 0x8080808080808080 are exactly the digits plus 128 (X < 2^60, so the
    // sum is an ordinary base-256 number without overflow).
    const uint32_t pt = threadIdx.x - 32 * kProdWarp0;   // one (b, c, dim) item per thread
    const uint32_t bcl = pt >> 3, il = pt & 7;             // local (b, c) row group, dim in chunk
    // the ciphertext value this thread encodes in chunk kc of unit u
    auto fetch = [&](uint64_t u, uint32_t kc) -> uint64_t {
      const Decoded D = decode_unit(u, N, A);
      const uint32_t bc = D.mt * 16 + bcl, i = kc * 8 + il;
      if (bc >= 2 * A.B || i >= A.d) return 0;
      const uint32_t b = bc >> 1, c = bc & 1;
      return __ldg(A.ct + ((((uint64_t)b * A.d + i) * 2 + c) * L + D.j) * N + D.s);
    };
    uint64_t g = 0;
    uint64_t X_next = blockIdx.x < A.units ? fetch(blockIdx.x, 0) : 0;
    for (uint64_t u = blockIdx.x; u < A.units && !abort_flag; u += gridDim.x) {
      const Decoded D = decode_unit(u, N, A);
      const uint64_t q = P.q[D.j];
      const uint64_t r256s = A.r256_shoup[D.j];
      bool ok = true;
      for (uint32_t kc = 0; kc < A.chunks; ++kc, ++g) {
        uint64_t X = X_next;
        if (kc + 1 < A.chunks) X_next = fetch(u, kc + 1);
        else if (u + gridDim.x < A.units) X_next = fetch(u + gridDim.x, 0);
        const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
        if (!mbar_wait(smem_u32(&bar_empty[st]), ph ^ 1, &abort_flag, A.err, 32)) { ok = false; break; }
        uint8_t* at = base + st * kStageBytes;
        uint32_t ylo[8], yhi[8];  // X 256^b8 mod q + 0x80..80, b8 = 0..7
#pragma unroll
        for (int b8 = 0; b8 < 8; ++b8) {
          const uint64_t y = X + 0x8080808080808080ull;
          ylo[b8] = (uint32_t)y;
          yhi[b8] = (uint32_t)(y >> 32);
          if (b8 < 7) X = mul_shoup(X, 256, r256s, q);
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const uint32_t sel = 0x7440u + (uint32_t)(a & 3);  // byte a, two zero bytes, 0x4B
          uint32_t w[4];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const uint32_t w0 = a < 4 ? ylo[2 * m] : yhi[2 * m];
            const uint32_t w1 = a < 4 ? ylo[2 * m + 1] : yhi[2 * m + 1];
            const float f0 = __uint_as_float(__byte_perm(w0, 0x4B000000u, sel)) - 8388736.0f;
            const float f1 = __uint_as_float(__byte_perm(w1, 0x4B000000u, sel)) - 8388736.0f;
            w[m] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
          }
          const uint32_t row = bcl * 8 + a;
          uint4* dst = reinterpret_cast<uint4*>(at + row * 128 + ((il ^ (row & 7)) << 4));
          *dst = make_uint4(w[0], w[1], w[2], w[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("bar.sync 1, %0;" ::"n"(kProdThreads) : "memory");
        if (pt == 0) mbar_arrive(smem_u32(&bar_full[st]));
      }
      if (!ok) break;
    }
  } else {
    // ---------------- epilogue ----------------
    // A warp reads 32 TMEM lanes (rows (b, c, a) of 4 row groups) x 16
    // columns, converts the exact fp32 sums to int32, transposes them through
    // shared memory so that each lane holds the 8 digit rows of one output,
    // and combines them exactly: lo = sum_{a<4} S_a 256^a and hi = sum_{a>=4}
    // S_a 256^(a-4) (both below 2^49 in magnitude), acc = lo + hi 2^32 mod q.
    const uint32_t ew = warp - kEpiWarp0;         // 0..7
    const uint32_t quarter = warp & 3;            // TMEM lanes 32 quarter ..
    const uint32_t half = ew >> 2;                // columns 128 half ..
    int32_t* trw = tr[ew];
    const uint32_t og = lane >> 3;                // output row group (0..3) of this lane
    const uint32_t oc = lane & 7;                 // output column within 8
    uint64_t r = 0;
    for (uint64_t u = blockIdx.x; u < A.units && !abort_flag; u += gridDim.x, ++r) {
      const uint32_t slot = (uint32_t)(r & 1), aph = (uint32_t)((r >> 1) & 1);
      if (!mbar_wait(smem_u32(&bar_tfull[slot]), aph, &abort_flag, A.err, 128)) break;
      tc_fence_after();
      const Decoded D = decode_unit(u, N, A);
      const uint64_t q = P.q[D.j];
      const uint64_t w32 = A.w32[D.j], w32s = A.w32_shoup[D.j];
      const uint32_t bc = D.mt * 16 + quarter * 4 + og;   // (b, c) of this lane's outputs
      const bool row_ok = bc < 2 * A.B;
      const uint32_t b = bc >> 1, c = bc & 1;
      uint64_t* orow = A.out + ((((uint64_t)b * A.K) * 2 + c) * L + D.j) * N + D.s;
      const uint64_t kstride = 2ull * L * N;
      for (uint32_t cc = 0; cc < 128 / kEpiCols; ++cc) {
        const uint32_t col0 = half * 128 + cc * kEpiCols;
        uint32_t v[kEpiCols];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + ((quarter * 32) << 16) + slot * kBN + col0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int x = 0; x < kEpiCols; ++x)
          trw[lane * kTrStride + x] = __float2int_rn(__uint_as_float(v[x]));
        __syncwarp();
#pragma unroll
        for (int h = 0; h < kEpiCols / 8; ++h) {
          const uint32_t col = h * 8 + oc;
          const int32_t* src = trw + (og * 8) * kTrStride + col;
          const int64_t lo = (int64_t)src[0] + ((int64_t)src[kTrStride] << 8) +
                             ((int64_t)src[2 * kTrStride] << 16) + ((int64_t)src[3 * kTrStride] << 24);
          const int64_t hi = (int64_t)src[4 * kTrStride] + ((int64_t)src[5 * kTrStride] << 8) +
                             ((int64_t)src[6 * kTrStride] << 16) + ((int64_t)src[7 * kTrStride] << 24);
          const uint64_t mu = A.mu64[D.j];
          const uint64_t rl = signed_mod(lo, q, mu);
          const uint64_t rh = signed_mod(hi, q, mu);
          const uint64_t res = add_mod(rl, mul_shoup(rh, w32, w32s, q), q);
          const uint32_t k = D.nt * kBN + col0 + col;
          if (row_ok && k < A.K) orow[(uint64_t)k * kstride] = res;
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_tempty[slot]));
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// Database digits: pt [K][L][d][N] u64 -> plimb [L][N][K][8 dpad] bf16, column
// 8 i + b = digit b of pt[k][j][i][s] (zero for i >= d).  One block per
// (k, j, 32-slot group) transposes through shared memory.
__global__ void prepare_limbs_kernel(const uint64_t* __restrict__ pt, uint32_t K, uint32_t L,
                                     uint32_t d, uint32_t dpad, uint32_t N,
                                     uint16_t* __restrict__ plimb) {
  extern __shared__ uint64_t tile[];  // [dpad][32]
  const uint32_t k = blockIdx.x, j = blockIdx.y, s0 = blockIdx.z * 32;
  for (uint32_t e = threadIdx.x; e < dpad * 32; e += blockDim.x) {
    const uint32_t i = e >> 5, s = e & 31;
    tile[e] = i < d ? pt[(((uint64_t)k * L + j) * d + i) * N + s0 + s] : 0;
  }
  __syncthreads();
  for (uint32_t e = threadIdx.x; e < dpad * 32; e += blockDim.x) {
    const uint32_t s = e / dpad, i = e % dpad;
    uint64_t y = tile[i * 32 + s];
    uint32_t w[4];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      int t = (int)(y & 255);
      y >>= 8;
      if (t >= 128) { t -= 256; y += 1; }
      const uint32_t h = __float_as_uint((float)t) >> 16;
      if (b & 1) w[b >> 1] |= h << 16;
      else w[b >> 1] = h;
    }
    uint16_t* dst = plimb + (((uint64_t)j * N + s0 + s) * K + k) * (8ull * dpad) + 8ull * i;
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

std::mutex g_encode_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encode(PFN_cuTensorMapEncodeTiled_v12000* out) {
  std::lock_guard<std::mutex> lock(g_encode_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  *out = g_encode;
  return cudaSuccess;
}

}  // namespace

size_t batched_limb_bytes(uint32_t L, uint32_t N, uint64_t K, uint32_t d) {
  const uint32_t dpad = (d + 7) / 8 * 8;
  return (size_t)L * N * K * 8ull * dpad * 2;
}

cudaError_t launch_prepare_limbs(const PrimeSet& P, const uint64_t* pt, uint64_t K, uint32_t d,
                                 uint16_t* plimb, cudaStream_t st) {
  const uint32_t dpad = (d + 7) / 8 * 8;
  const size_t smem = sizeof(uint64_t) * dpad * 32;
  cudaError_t e = cudaFuncSetAttribute(prepare_limbs_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)K, P.L, P.N / 32);
  prepare_limbs_kernel<<<grid, 256, smem, st>>>(pt, (uint32_t)K, P.L, d, dpad, P.N, plimb);
  return cudaGetLastError();
}

int make_limb_map(const PrimeSet& P, const uint16_t* plimb, uint64_t K, uint32_t d, void* map_out) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  cudaError_t e = get_encode(&enc);
  if (e != cudaSuccess) return cuda_fail(e, "cuTensorMapEncodeTiled entry point");
  const uint32_t dpad = (d + 7) / 8 * 8;
  const cuuint64_t dims[3] = {8ull * dpad, K, (cuuint64_t)P.L * P.N};
  const cuuint64_t strides[2] = {8ull * dpad * 2, K * 8ull * dpad * 2};
  const cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)kBN, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                   const_cast<uint16_t*>(plimb), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SANNS_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return SANNS_OK;
}

cudaError_t launch_batched_mac(const PrimeSet& P, const void* map, const uint64_t* ct, uint32_t B,
                               uint32_t d, uint64_t K, uint64_t* out, int* err, int sms,
                               cudaStream_t st) {
  BatchArgs A;
  memset(&A, 0, sizeof(A));
  A.ct = ct;
  A.out = out;
  A.err = err;
  A.B = B;
  A.d = d;
  A.dpad = (d + 7) / 8 * 8;
  A.K = (uint32_t)K;
  A.MT = (2 * B + 15) / 16;
  A.NT = (uint32_t)((K + kBN - 1) / kBN);
  A.chunks = A.dpad / 8;
  A.units = (uint64_t)P.L * P.N * A.NT * A.MT;
  for (uint32_t j = 0; j < P.L; ++j) {
    uint64_t w = 1 % P.q[j];
    for (int a = 0; a < 8; ++a) {
      A.w256[j][a] = w;
      A.w256_shoup[j][a] = shoup_of(w, P.q[j]);
      w = (uint64_t)(((u128)w * 256) % P.q[j]);
    }
    A.r256_shoup[j] = shoup_of(256 % P.q[j], P.q[j]);
    A.w32[j] = (uint64_t)(((u128)1 << 32) % P.q[j]);
    A.w32_shoup[j] = shoup_of(A.w32[j], P.q[j]);
    A.mu64[j] = (uint64_t)(((u128)1 << 64) / P.q[j]);
  }
  const size_t smem = (size_t)kStages * kStageBytes + 1024;
  cudaError_t e = cudaFuncSetAttribute(batched_mac_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  uint64_t grid = (uint64_t)(sms > 0 ? sms : 148);
  if (grid > A.units) grid = A.units;
  CUtensorMap m;
  memcpy(&m, map, sizeof(m));
  batched_mac_kernel<<<(unsigned)grid, kThreads, smem, st>>>(m, P, A);
  return cudaGetLastError();
}

}  // namespace sanns
