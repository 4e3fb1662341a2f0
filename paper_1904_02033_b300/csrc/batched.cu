// K5: the batched ct x pt MAC on the tensor cores (tcgen05, kind::f16, fp16
// operands, fp32 accumulation in TMEM), exact.
//
// With B queries, every (prime j, slot s) is the contraction
//     C[(b, c)][k] = sum_i A[(b, c)][i] P[k][i]  mod q_j,
// A = the query ciphertexts (NTT form), P = the encoded database.  Residues
// are split into balanced base-256 digits in [-128, 127], which fp16 holds
// exactly.  The database side is split once, P[k][i] = sum_b p_b 256^b; the
// query side is folded with the digit weight of the database side,
// X_b = A 256^b mod q = sum_a x_{b,a} 256^a, so that
//     C = sum_a 256^a S_a,   S_a = sum_{i, b} x_{b,a}[i] p_b[k][i]   (mod q).
// S_a is one GEMM with rows (b, c, a), columns k and contraction (i, b):
// every product is at most 2^14 in magnitude and a sum of 8 d <= 1024 of them
// stays within 2^24, so the fp32 accumulation is exact for d <= 128.
//
// The GEMM is laid out with the database on the M side: rows are blocks k
// (128 per tile, read by TMA from the resident digit layout), columns are
// (b, c, a) for 16 queries (256 per tile, generated in shared memory), so one
// TMEM lane holds the 8 digit sums S_0..S_7 of an output in 8 consecutive
// columns and the epilogue needs no data exchange between lanes.
//
// One persistent CTA per SM, warp-specialised (18 warps):
//   warp 0      TMA producer: database digit tile (128 rows x 64 fp16) per
//               stage, and an L2 prefetch of a later unit's tiles
//   warp 1      TMEM owner and MMA issuer (one thread): 4 MMAs of
//               M = 128, N = 256, K = 16 per stage
//   warps 2-9   query-digit producers: 256 rows x 64 fp16 per stage, written
//               into shared memory in the 128-byte swizzled layout
//   warps 10-17 epilogue: TMEM -> registers, exact int64 combination of each
//               output's 8 digit sums, one mod-q step, store acc[b][k][c][j][s]
// Work unit = (prime, slot, 128-block K tile, 16-query Q tile), Q tile
// fastest, so the CTAs running side by side share each database tile
// through L2.
// Every wait is bounded: on time-out the kernel raises a device error flag,
// drains its own copies, frees TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "internal.h"

namespace sanns {

namespace {

constexpr int kStages = 4;
constexpr int kBM = 128;                 // database blocks per tile (A operand, TMA)
constexpr int kBN = 256;                 // query rows (b, c, a) per tile: 32 (b, c) x 8 digits
constexpr int kBK = 64;                  // contraction columns (8 dims x 8 digits) per stage
constexpr int kQG = kBN / 8;             // (b, c) row groups per tile
constexpr int kATile = kBM * kBK * 2;    // 16 KB
constexpr int kBTile = kBN * kBK * 2;    // 32 KB
constexpr int kStageBytes = kATile + kBTile;
constexpr int kProdWarp0 = 2;
constexpr int kProdWarps = 8;
constexpr int kProdThreads = 32 * kProdWarps;
static_assert(kProdThreads == kQG * 8, "one (row group, dimension) item per producer thread");
constexpr int kEpiWarp0 = kProdWarp0 + kProdWarps;    // 10
constexpr int kEpiWarps = 8;                          // two per TMEM lane quarter
constexpr int kThreads = 32 * (kEpiWarp0 + kEpiWarps);  // 576
constexpr unsigned long long kWaitCycles = 4ull << 30;  // ~2 s at 2 GHz

struct BatchArgs {
  const uint64_t* xm;     // [S][2B][dpad][8]: query values times 256^b mod q, slot range
  uint32_t s_begin, s_count;
  uint64_t* out;          // [B][K][2][L][N]
  int* err;               // device error word
  uint32_t B, d, dpad, K;
  uint32_t QT, KT, chunks;
  uint64_t units;
  uint64_t w256[kMaxPrimes][8];        // 256^a mod q_j
  uint64_t w256_shoup[kMaxPrimes][8];
  uint64_t r256_shoup[kMaxPrimes];     // Shoup companion of 256
  uint64_t w32[kMaxPrimes];            // 2^32 mod q_j
  uint64_t w32_shoup[kMaxPrimes];
  uint64_t mu64[kMaxPrimes];           // floor(2^64 / q_j)
  // wait back-off (ns) per role; how many of its own units ahead a CTA
  // prefetches the database and query tiles into L2 (0: none)
  uint32_t sleep_tma, sleep_mma, sleep_prod, sleep_epi, prefetch_units;
  const uint16_t* plimb;  // [L][N][K][8 dpad] database digits (prefetch addresses)
  uint64_t lo_bias[kMaxPrimes];  // a multiple of q_j at or above 2^49
};

// L2 prefetch of [p, p + bytes) in pieces of at most 32 KB (16-byte aligned
// address and size).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  const char* c = static_cast<const char*>(p);
  for (uint32_t off = 0; off < bytes; off += 32768) {
    const uint32_t n = bytes - off < 32768 ? bytes - off : 32768;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + off), "r"(n) : "memory");
  }
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

// kind::f16: D fp32, A and B fp16 (format 0), both K-major, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
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
  uint32_t j, qt, kt, s, sl;
};

// unit = ((j S + s') KT + kt) QT + qt over the launch's slot range s' in
// [0, s_count): the query tiles of one database tile are consecutive, so CTAs
// running side by side share it through L2.  D.s is the absolute slot and
// D.sl the slot within the range.  Units fit in 32 bits (the launcher checks).
__device__ __forceinline__ Decoded decode_unit(uint32_t u, uint32_t logN, const BatchArgs& A) {
  Decoded D;
  D.qt = u % A.QT;
  uint32_t r = u / A.QT;
  D.kt = r % A.KT;
  r /= A.KT;
  D.sl = r % A.s_count;
  D.s = A.s_begin + D.sl;
  D.j = r / A.s_count;
  (void)logN;
  return D;
}


__global__ void __launch_bounds__(kThreads, 1)
batched_mac_kernel(const __grid_constant__ CUtensorMap pmap, PrimeSet P, BatchArgs A) {
  extern __shared__ __align__(1024) uint8_t dsmem[];
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages];
  __shared__ __align__(8) uint64_t bar_tfull[2], bar_tempty[2];
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;

  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* base = dsmem + ((1024 - (smem_u32(dsmem) & 1023)) & 1023);
  const uint32_t sbase = smem_u32(base);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1 + kProdWarps);
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
    // the whole warp walks the loop (converged); lane 0 waits and issues
    uint64_t g = 0;
    bool ok = true;
    for (uint64_t u = blockIdx.x; u < A.units && ok; u += gridDim.x) {
      const Decoded D = decode_unit((uint32_t)u, P.logN, A);
      const uint64_t pu = u + (uint64_t)A.prefetch_units * gridDim.x;
      if (lane == 0 && A.prefetch_units && pu < A.units) {
        // database tile (rows kt*128 .. of slot (j, s)) and query multiples
        // (row groups qt*32 .. of slot (j, s')) of a later unit of this CTA
        const Decoded F = decode_unit((uint32_t)pu, P.logN, A);
        const uint32_t rows = A.K - F.kt * kBM < (uint32_t)kBM ? A.K - F.kt * kBM : (uint32_t)kBM;
        prefetch_l2(A.plimb + (((uint64_t)F.j * N + F.s) * A.K + (uint64_t)F.kt * kBM) * 8 * A.dpad,
                    rows * 16u * A.dpad);
        const uint32_t twoB = 2 * A.B, bc0 = F.qt * kQG;
        const uint32_t groups = twoB - bc0 < (uint32_t)kQG ? twoB - bc0 : (uint32_t)kQG;
        prefetch_l2(A.xm + (((uint64_t)F.j * A.s_count + F.sl) * twoB + bc0) * A.dpad * 8,
                    groups * 64u * A.dpad);
      }
      for (uint32_t kc = 0; kc < A.chunks; ++kc, ++g) {
        const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
        bool ready = true;
        if (lane == 0) ready = mbar_wait(smem_u32(&bar_empty[st]), ph ^ 1, &abort_flag, A.err, A.sleep_tma);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { ok = false; break; }
        if (lane == 0) {
          const uint32_t full = smem_u32(&bar_full[st]);
          mbar_arrive_tx(full, kATile);
          tma_load_3d(sbase + st * kStageBytes, &pmap, (int)(kc * kBK), (int)(D.kt * kBM),
                      (int)(D.j * N + D.s), full);
        }
        __syncwarp();
      }
    }
    // drain: every issued copy completes before the CTA may exit
    if (!ok && lane == 0) {
      const uint64_t first = g > kStages ? g - kStages : 0;
      for (uint64_t h = first; h < g; ++h) {
        const uint32_t st = (uint32_t)(h % kStages), ph = (uint32_t)((h / kStages) & 1);
        const unsigned long long t0 = clock64();
        while (!mbar_try(smem_u32(&bar_full[st]), ph) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    // the whole warp walks the loop (converged); lane 0 waits and issues
    uint64_t g = 0, r = 0;
    bool ok = true;
    for (uint64_t u = blockIdx.x; u < A.units && ok; u += gridDim.x, ++r) {
      const uint32_t slot = (uint32_t)(r & 1), aph = (uint32_t)((r >> 1) & 1);
      bool ready = true;
      if (lane == 0) ready = mbar_wait(smem_u32(&bar_tempty[slot]), aph ^ 1, &abort_flag, A.err, A.sleep_mma);
      if (!__shfl_sync(0xffffffffu, (int)ready, 0)) break;
      tc_fence_after();
      const uint32_t dt = tmem + slot * kBN;
      for (uint32_t kc = 0; kc < A.chunks; ++kc, ++g) {
        const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
        if (lane == 0) ready = mbar_wait(smem_u32(&bar_full[st]), ph, &abort_flag, A.err, A.sleep_mma);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { ok = false; break; }
        tc_fence_after();
        if (lane == 0) {
          const uint32_t a_addr = sbase + st * kStageBytes, b_addr = a_addr + kATile;
          const uint64_t ad = smem_desc(a_addr), bd = smem_desc(b_addr);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k)
            mma_f16(dt, ad + 2 * k, bd + 2 * k, (kc > 0 || k > 0) ? 1u : 0u);
          mma_commit(smem_u32(&bar_empty[st]));
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma_commit(smem_u32(&bar_tfull[slot]));
      __syncwarp();
    }
  } else if (warp < kEpiWarp0) {
    // ---------------- query-digit producers ----------------
    // The pre-kernel stored, for every query value, Y_b = X 256^b mod q +
    // 0x8080808080808080 (b = 0..7), whose bytes are the balanced base-256
    // digits of X 256^b plus 128, with the bytes of Y_2m and Y_2m+1
    // interleaved (byte 2a of pair m = byte a of Y_2m, byte 2a + 1 = byte a
    // of Y_2m+1).  Row a of the tile takes bytes 2a, 2a + 1 of every pair: one
    // byte permute puts them under the fp16 exponent of 1024 (0x64vv = 1024 +
    // v, exact) and one f16x2 subtraction of 1152 leaves the digits.
    const uint32_t pt = threadIdx.x - 32 * kProdWarp0;   // one (b, c, dim) item per thread
    const uint32_t bcl = pt >> 3, il = pt & 7;             // (b, c) row group in tile, dim in chunk
    const uint32_t units = (uint32_t)A.units, chunks = A.chunks;
    const uint32_t twoB = 2 * A.B;
    // this thread's 8 values of chunk 0 in unit u (null past the units or 2B)
    auto unit_base = [&](uint32_t u) -> const ulonglong2* {
      if (u >= units) return nullptr;
      const Decoded D = decode_unit(u, P.logN, A);
      const uint32_t bc = D.qt * kQG + bcl;
      if (bc >= twoB) return nullptr;
      return reinterpret_cast<const ulonglong2*>(
          A.xm + ((((uint64_t)D.j * A.s_count + D.sl) * twoB + bc) * A.dpad + il) * 8);
    };
    // chunk k advances the dimension by 8: 8 items x 64 bytes; an item past d
    // or past 2B holds Y_b = 0x80.. (all digits zero)
    auto load_item = [&](const ulonglong2* b0, uint32_t k, ulonglong2 (&dst)[4]) {
      const bool v = b0 != nullptr && k * 8 + il < A.d;
#pragma unroll
      for (int h = 0; h < 4; ++h)
        dst[h] = v ? __ldg(b0 + 32 * k + h) : make_ulonglong2(0x8080808080808080ull, 0x8080808080808080ull);
    };
    // Each warp fills its own 32 items (4 row groups x 8 dims) of every stage
    // and arrives on the stage's barrier itself, so warps run ahead of one
    // another; values are prefetched two chunks ahead.
    uint32_t fu = blockIdx.x, fk = 0;
    const ulonglong2* fb = unit_base(fu);
    auto advance = [&]() {
      if (++fk == chunks) { fk = 0; fu += gridDim.x; fb = unit_base(fu); }
    };
    ulonglong2 nx0[4], nx1[4];
    load_item(fb, fk, nx0);
    advance();
    load_item(fb, fk, nx1);
    advance();
    uint64_t g = 0;
    uint32_t cu = blockIdx.x, ck = 0;
    while (cu < units) {
      ulonglong2 cur[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) { cur[h] = nx0[h]; nx0[h] = nx1[h]; }
      load_item(fb, fk, nx1);
      advance();
      const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
      ++g;
      // lane 0 polls the stage, the warp follows its decision
      bool ready = true;
      if (lane == 0) ready = mbar_wait(smem_u32(&bar_empty[st]), ph ^ 1, &abort_flag, A.err, A.sleep_prod);
      if (!__shfl_sync(0xffffffffu, (int)ready, 0)) break;
      uint8_t* at = base + st * kStageBytes + kATile;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const uint32_t sel = (a & 1) ? 0x4342u : 0x4140u;
        uint32_t w[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const uint64_t z = (a >> 1) < 2 ? cur[m].x : cur[m].y;
          const uint32_t zw = ((a >> 1) & 1) ? (uint32_t)(z >> 32) : (uint32_t)z;
          const uint32_t hv = __byte_perm(zw, 0x64646464u, sel);
          uint32_t h;
          asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(h) : "r"(hv), "r"(0x64806480u));
          w[m] = h;
        }
        const uint32_t row = bcl * 8 + a;
        uint4* dst = reinterpret_cast<uint4*>(at + row * 128 + ((il ^ (row & 7)) << 4));
        *dst = make_uint4(w[0], w[1], w[2], w[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_full[st]));
      if (++ck == chunks) { ck = 0; cu += gridDim.x; }
    }
  } else {
    // ---------------- epilogue ----------------
    // Lane = database block k of the tile; columns (bc, a) with a fastest, so
    // each x32 load holds the 8 digit sums of 4 outputs.  Exact combination:
    // lo = sum_{a<4} S_a 256^a and hi = sum_{a>=4} S_a 256^(a-4) (both below
    // 2^49 in magnitude), acc = lo + hi 2^32 mod q.
    const uint32_t quarter = warp & 3;            // TMEM lanes 32 quarter ..
    const uint32_t chalf = (warp - kEpiWarp0) >> 2;  // column half of the tile
    uint64_t r = 0;
    for (uint64_t u = blockIdx.x; u < A.units && !abort_flag; u += gridDim.x, ++r) {
      const uint32_t slot = (uint32_t)(r & 1), aph = (uint32_t)((r >> 1) & 1);
      // lane 0 waits for the accumulator, the warp follows its decision
      bool ready = true;
      if (lane == 0) ready = mbar_wait(smem_u32(&bar_tfull[slot]), aph, &abort_flag, A.err, A.sleep_epi);
      if (!__shfl_sync(0xffffffffu, (int)ready, 0)) break;
      tc_fence_after();
      const Decoded D = decode_unit((uint32_t)u, P.logN, A);
      const uint64_t q = P.q[D.j], mu = A.mu64[D.j];
      const int64_t bias = (int64_t)A.lo_bias[D.j];
      const uint64_t w32 = A.w32[D.j], w32s = A.w32_shoup[D.j];
      const uint32_t k = D.kt * kBM + quarter * 32 + lane;
      const bool k_ok = k < A.K;
      for (uint32_t cc = chalf * (kBN / 64); cc < (chalf + 1) * (kBN / 64); ++cc) {
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, "
            "%27, %28, %29, %30, %31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
              "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
              "=r"(v[30]), "=r"(v[31])
            : "r"(tmem + ((quarter * 32) << 16) + slot * kBN + cc * 32));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          int32_t sa[8];
#pragma unroll
          for (int a = 0; a < 8; ++a) sa[a] = __float2int_rn(__uint_as_float(v[o * 8 + a]));
          const int64_t lo = (int64_t)sa[0] + (int64_t)sa[1] * 256 + (int64_t)sa[2] * 65536 +
                             (int64_t)sa[3] * 16777216;
          const int64_t hi = (int64_t)sa[4] + (int64_t)sa[5] * 256 + (int64_t)sa[6] * 65536 +
                             (int64_t)sa[7] * 16777216;
          // |lo|, |hi| < 2^49 <= bias: both biased values are positive and
          // below 2^50 + q; hi 2^32 lazily below 2q, the sum below 2^64
          const uint64_t hs = mul_shoup_lazy((uint64_t)(hi + bias), w32, w32s, q);
          const uint64_t res = mod_t64(hs + (uint64_t)(lo + bias), q, mu);
          const uint32_t bc = D.qt * kQG + cc * 4 + o;
          if (k_ok && bc < 2 * A.B) {
            const uint32_t b = bc >> 1, c = bc & 1;
            A.out[((((uint64_t)b * A.K + k) * 2 + c) * L + D.j) * N + D.s] = res;
          }
        }
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

// Database digits: pt [K][L][d][N] u64 -> plimb [L][N][K][8 dpad] fp16, column
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
      const uint32_t h = (uint32_t)__half_as_ushort(__float2half_rn((float)t));
      if (b & 1) w[b >> 1] |= h << 16;
      else w[b >> 1] = h;
    }
    uint16_t* dst = plimb + (((uint64_t)j * N + s0 + s) * K + k) * (8ull * dpad) + 8ull * i;
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// X_b = ct 256^b mod q for b = 0..7, for the slots [s_begin, s_begin + S):
// xm[j][s'][bc][i][8 words], bc = 2 b_query + c, stored as the biased and
// pairwise byte-interleaved form the digit producers read.  One thread per (j, s', bc, i),
// slot fastest so that the ciphertext reads coalesce.
__global__ void expand_query_kernel(PrimeSet P, const uint64_t* __restrict__ ct, uint32_t B,
                                    uint32_t d, uint32_t dpad, uint32_t s_begin, uint32_t S,
                                    const uint64_t* __restrict__ w256,
                                    const uint64_t* __restrict__ w256s,
                                    uint64_t* __restrict__ xm) {
  const uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t total = (uint64_t)P.L * S * 2 * B * d;
  if (gid >= total) return;
  const uint32_t sl = (uint32_t)(gid % S);
  uint64_t r = gid / S;
  const uint32_t i = (uint32_t)(r % d);
  r /= d;
  const uint32_t bc = (uint32_t)(r % (2 * B));
  const uint32_t j = (uint32_t)(r / (2 * B));
  const uint32_t b = bc >> 1, c = bc & 1;
  const uint32_t N = P.N, L = P.L;
  const uint64_t q = P.q[j];
  const uint64_t X = ct[((((uint64_t)b * d + i) * 2 + c) * L + j) * N + s_begin + sl];
  uint64_t v[8];
  v[0] = X;
#pragma unroll
  for (int k = 1; k < 8; ++k) v[k] = mul_shoup(X, w256[j * 8 + k], w256s[j * 8 + k], q);
  ulonglong2* dst = reinterpret_cast<ulonglong2*>(
      xm + ((((uint64_t)j * S + sl) * 2 * B + bc) * dpad + i) * 8);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    // + 0x80 per byte (no carry out: X < 2^62), then bytes of the pair interleaved
    const uint64_t y0 = v[2 * m] + 0x8080808080808080ull, y1 = v[2 * m + 1] + 0x8080808080808080ull;
    const uint32_t l0 = (uint32_t)y0, h0 = (uint32_t)(y0 >> 32), l1 = (uint32_t)y1, h1 = (uint32_t)(y1 >> 32);
    const uint64_t zx = (uint64_t)__byte_perm(l0, l1, 0x5140) | ((uint64_t)__byte_perm(l0, l1, 0x7362) << 32);
    const uint64_t zy = (uint64_t)__byte_perm(h0, h1, 0x5140) | ((uint64_t)__byte_perm(h0, h1, 0x7362) << 32);
    dst[m] = make_ulonglong2(zx, zy);
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
  const cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)kBM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3,
                   const_cast<uint16_t*>(plimb), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SANNS_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return SANNS_OK;
}

cudaError_t launch_batched_mac(const PrimeSet& P, const void* map, const uint16_t* plimb,
                               const uint64_t* ct, uint32_t B,
                               uint32_t d, uint64_t K, uint64_t* out, int* err, int sms,
                               const uint32_t tune[6], cudaStream_t st) {
  BatchArgs A;
  memset(&A, 0, sizeof(A));
  A.sleep_tma = tune[0];
  A.sleep_mma = tune[1];
  A.sleep_prod = tune[2];
  A.sleep_epi = tune[3];
  A.prefetch_units = tune[4];
  A.plimb = plimb;
  A.out = out;
  A.err = err;
  A.B = B;
  A.d = d;
  A.dpad = (d + 7) / 8 * 8;
  A.K = (uint32_t)K;
  A.QT = (2 * B + kQG - 1) / kQG;
  A.KT = (uint32_t)((K + kBM - 1) / kBM);
  A.chunks = A.dpad / 8;
  uint64_t hw[kMaxPrimes * 16];
  for (uint32_t j = 0; j < P.L; ++j) {
    uint64_t w = 1 % P.q[j];
    for (int a = 0; a < 8; ++a) {
      A.w256[j][a] = w;
      A.w256_shoup[j][a] = shoup_of(w, P.q[j]);
      hw[j * 8 + a] = w;
      hw[kMaxPrimes * 8 + j * 8 + a] = A.w256_shoup[j][a];
      w = (uint64_t)(((u128)w * 256) % P.q[j]);
    }
    A.r256_shoup[j] = shoup_of(256 % P.q[j], P.q[j]);
    A.w32[j] = (uint64_t)(((u128)1 << 32) % P.q[j]);
    A.w32_shoup[j] = shoup_of(A.w32[j], P.q[j]);
    A.mu64[j] = (uint64_t)(((u128)1 << 64) / P.q[j]);
    A.lo_bias[j] = ((1ull << 49) + P.q[j] - 1) / P.q[j] * P.q[j];
  }
  // slot ranges bound the scratch of the query multiples (tune[5] MiB, at
  // least one slot)
  const uint64_t per_slot = (uint64_t)P.L * 2 * B * A.dpad * 8 * sizeof(uint64_t);
  uint64_t S = ((uint64_t)tune[5] << 20) / per_slot;
  if (S < 1) S = 1;
  if (S > P.N) S = P.N;
  const size_t smem = (size_t)kStages * kStageBytes + 1024;
  cudaError_t e = cudaFuncSetAttribute(batched_mac_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  uint64_t* scratch = nullptr;
  e = cudaMallocAsync(&scratch, per_slot * S + sizeof(hw), st);
  if (e != cudaSuccess) return e;
  uint64_t* dw = scratch + per_slot * S / sizeof(uint64_t);
  e = cudaMemcpyAsync(dw, hw, sizeof(hw), cudaMemcpyHostToDevice, st);
  CUtensorMap m;
  memcpy(&m, map, sizeof(m));
  for (uint64_t s0 = 0; s0 < P.N && e == cudaSuccess; s0 += S) {
    const uint32_t cnt = (uint32_t)(s0 + S <= P.N ? S : P.N - s0);
    A.s_begin = (uint32_t)s0;
    A.s_count = cnt;
    A.xm = scratch;
    A.units = (uint64_t)P.L * cnt * A.KT * A.QT;
    if (A.units >= (1ull << 31)) { e = cudaErrorInvalidValue; break; }
    const uint64_t threads = (uint64_t)P.L * cnt * 2 * B * d;
    expand_query_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        P, ct, B, d, A.dpad, (uint32_t)s0, cnt, dw, dw + kMaxPrimes * 8, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    uint64_t grid = (uint64_t)(sms > 0 ? sms : 148);
    if (grid > A.units) grid = A.units;
    batched_mac_kernel<<<(unsigned)grid, kThreads, smem, st>>>(m, P, A);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(scratch, st);
  return e != cudaSuccess ? e : e2;
}

}  // namespace sanns
