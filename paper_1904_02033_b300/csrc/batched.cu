// K5: the batched ct x pt MAC on the tensor cores (tcgen05, kind::f16, fp16
// operands, fp32 accumulation in TMEM), exact: the sum_i CMult(c_i, g_ik) of
// the linear-scan protocol's step 3 (Sec. 5.3) for many queries at once.
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
// stages + the epilogue's held first slot of a pair (16 outputs per thread)
constexpr int kSmem1 = kStages * kStageBytes + 16 * 32 * kEpiWarps * 8 + 1024;
constexpr unsigned long long kWaitCycles = 4ull << 30;  // ~2 s at 2 GHz

struct BatchArgs {
  const uint64_t* xm;     // query multiples of the slot range, layout of expand_query_kernel
  uint32_t s_begin, s_count;
  uint64_t* out;          // [B][K][2][L][N]
  uint32_t out16;         // out is 16-byte aligned (paired stores)
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
  // TMA-fed query digits: [L S'][16 B][8 dpad] fp16 rows (bc, a) of the slot
  // range (see expand_query_f16_kernel), for the prefetch addresses
  const uint16_t* xh;
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

// Bounded wait; false when the CTA is aborting or the wait timed out after
// limit_cycles (which also raises the abort flag and the device error word).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, uint32_t sleep_ns = 0,
                                          unsigned long long limit_cycles = kWaitCycles) {
  const unsigned long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (sleep_ns && it > 2) __nanosleep(sleep_ns);
    if ((it & 255) == 255) {
      if (*abort_flag) return false;
      if (clock64() - t0 > limit_cycles) {
        *abort_flag = 1;
        atomicExch(err, SANNS_ETIMEOUT);
        return false;
      }
    }
  }
}

// Self-test of the time-out path: one thread waits, through mbar_wait, on a
// barrier that nothing arrives on, so the wait gives up after limit_cycles,
// raises the device error word and the kernel returns.
__global__ void wait_selftest_kernel(int* err, unsigned long long limit_cycles) {
  __shared__ alignas(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, &abort_flag, err, 1000, limit_cycles);
  __syncthreads();
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


// Digit rows of one (b, c, dimension) item into a swizzled B stage: row
// 8 bcl + a holds digit a of the item's eight multiples (columns 8 il .. 8 il
// + 7 of the 64-column stage).  cur = the pre-kernel's biased, pairwise
// byte-interleaved multiples (see expand_query_kernel).
__device__ __forceinline__ void store_digit_rows(uint8_t* at, uint32_t bcl, uint32_t il,
                                                 const ulonglong2 (&cur)[4]) {
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
}

// One 32-column TMEM load of the epilogue: columns (bc, a) with a fastest hold
// the 8 digit sums of 4 outputs.  Exact combination: lo = sum_{a<4} S_a 256^a
// and hi = sum_{a>=4} S_a 256^(a-4) (both below 2^49 in magnitude), acc = lo +
// hi 2^32 mod q, returned in res[0 .. 3].
__device__ __forceinline__ void epilogue_values(uint32_t taddr, const BatchArgs& A, const PrimeSet& P,
                                                const Decoded& D, uint64_t (&res)[4]) {
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
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  const uint64_t q = P.q[D.j], mu = A.mu64[D.j];
  const int64_t bias = (int64_t)A.lo_bias[D.j];
  const uint64_t w32 = A.w32[D.j], w32s = A.w32_shoup[D.j];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    int32_t sa[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) sa[a] = __float2int_rn(__uint_as_float(v[o * 8 + a]));
    const int64_t lo = (int64_t)sa[0] + (int64_t)sa[1] * 256 + (int64_t)sa[2] * 65536 +
                       (int64_t)sa[3] * 16777216;
    const int64_t hi = (int64_t)sa[4] + (int64_t)sa[5] * 256 + (int64_t)sa[6] * 65536 +
                       (int64_t)sa[7] * 16777216;
    // |lo|, |hi| < 2^49 <= bias: both biased values are positive and below
    // 2^50 + q; hi 2^32 lazily below 2q, the sum below 2^64
    const uint64_t hs = mul_shoup_lazy((uint64_t)(hi + bias), w32, w32s, q);
    res[o] = mod_t64(hs + (uint64_t)(lo + bias), q, mu);
  }
}

// epilogue_values, then one 8-byte store per output of slot D.s; bc0 = the
// (b, c) row of the first of the 4 outputs.
__device__ __forceinline__ void epilogue_chunk(uint32_t taddr, const BatchArgs& A, const PrimeSet& P,
                                               const Decoded& D, uint32_t k, bool k_ok,
                                               uint32_t bc0) {
  uint64_t res[4];
  epilogue_values(taddr, A, P, D, res);
  const uint32_t N = P.N, L = P.L;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const uint32_t bc = bc0 + o;
    if (k_ok && bc < 2 * A.B) {
      const uint32_t b = bc >> 1, c = bc & 1;
      A.out[((((uint64_t)b * A.K + k) * 2 + c) * L + D.j) * N + D.s] = res[o];
    }
  }
}

// Unit m of this CTA for the single-SM tile: pairs of slots, both halves back
// to back, so the epilogue can store both slots of an output as one 16-byte
// word.  Pair p = blockIdx.x + (m / 2) gridDim.x over A.units pairs, decoded
// as ((j S/2 + s'/2) KT + kt) QT + qt; half m % 2 gives slot s' = 2 (s'/2) +
// m % 2.  False past the last pair.
//
// With clusters of CL CTAs (CL > 1), pairs are counted per cluster: pair p =
// cluster + (m / 2) (clusters in the grid) over A.units pairs, whose database
// tile index counts groups of CL tiles; the CTA of rank r takes tile
// CL group + r, so the CTAs of a cluster share the slot and the query tile.
template <int CL>
__device__ __forceinline__ bool unit_of(uint32_t m, const BatchArgs& A, Decoded& D) {
  const uint32_t cid = blockIdx.x / CL, rank = blockIdx.x % CL, ncl = gridDim.x / CL;
  const uint64_t p = cid + (uint64_t)(m >> 1) * ncl;
  if (p >= A.units) return false;
  const uint32_t half = A.s_count >> 1;
  const uint32_t ktg = A.KT / CL;
  uint32_t r = (uint32_t)p;
  D.qt = r % A.QT;
  r /= A.QT;
  D.kt = (r % ktg) * CL + rank;
  r /= ktg;
  D.sl = 2 * (r % half) + (m & 1);
  D.s = A.s_begin + D.sl;
  D.j = r / half;
  return true;
}

__device__ __forceinline__ void tma_load_3d_mc(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                               uint32_t bar, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar), "h"(mask)
      : "memory");
}

// completion of this thread's prior MMAs arrives on the barrier at the same
// offset in every CTA of `mask` (single-CTA MMAs)
__device__ __forceinline__ void mma_commit_mc1(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar), "h"(mask)
      : "memory");
}

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

__device__ __forceinline__ bool mbar_try_acq_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on a barrier that other CTAs of the cluster arrive on
// (cluster-scope acquire), otherwise as mbar_wait.
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                                  int* err, uint32_t sleep_ns = 0) {
  const unsigned long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_acq_cluster(bar, parity)) return true;
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

// TMA_B: the query-digit tile of every stage arrives by TMA from the fp16
// rows written by expand_query_f16_kernel (xmap), and the producer warps stay
// idle; otherwise they generate it from the byte-interleaved multiples.
//
// CL > 1 (with TMA_B): clusters of CL CTAs take CL consecutive database tiles
// of the same slot and query tile; each CTA loads 256 / CL of the query-digit
// rows with cluster multicast, so every CTA receives the whole query tile
// while the cluster reads it from L2 once.  A stage is then free only once
// every CTA of the cluster has consumed it: the MMA completion arrives on the
// stage-empty barrier of all CL CTAs.
template <bool TMA_B, int CL>
__global__ void __launch_bounds__(kThreads, 1)
batched_mac_kernel(const __grid_constant__ CUtensorMap pmap, const __grid_constant__ CUtensorMap xmap,
                   PrimeSet P, BatchArgs A) {
  static_assert(CL == 1 || TMA_B, "clusters share TMA-fed query tiles");
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
      mbar_init(smem_u32(&bar_full[s]), TMA_B ? 1 : 1 + kProdWarps);
      mbar_init(smem_u32(&bar_empty[s]), CL);
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
  if (CL > 1) cluster_barrier();  // every CTA's barriers exist before any multicast
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;
  const uint32_t N = P.N;
  const uint32_t crank = blockIdx.x % CL;
  constexpr uint16_t kMask = (uint16_t)((1u << CL) - 1);

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    // the whole warp walks the loop (converged); lane 0 waits and issues
    uint64_t g = 0;
    bool ok = true;
    for (uint32_t m = 0; ok; ++m) {
      Decoded D, F;
      if (!unit_of<CL>(m, A, D)) break;
      if (lane == 0 && A.prefetch_units && unit_of<CL>(m + 2 * A.prefetch_units, A, F) &&
          F.kt * kBM < A.K) {
        // database tile (rows kt*128 .. of slot (j, s)) and query multiples
        // (row groups qt*32 .. of slot (j, s')) of a later unit of this CTA
        const uint32_t rows = A.K - F.kt * kBM < (uint32_t)kBM ? A.K - F.kt * kBM : (uint32_t)kBM;
        prefetch_l2(A.plimb + (((uint64_t)F.j * N + F.s) * A.K + (uint64_t)F.kt * kBM) * 8 * A.dpad,
                    rows * 16u * A.dpad);
        const uint32_t twoB = 2 * A.B, bc0 = F.qt * kQG;
        const uint32_t groups = twoB - bc0 < (uint32_t)kQG ? twoB - bc0 : (uint32_t)kQG;
        if (TMA_B)
          prefetch_l2(A.xh + (((uint64_t)F.j * A.s_count + F.sl) * 8 * twoB + 8 * bc0) * 8 * A.dpad,
                      groups * 128u * A.dpad);
        else
          prefetch_l2(A.xm + (((uint64_t)F.j * A.s_count + F.sl) * twoB + bc0) * A.dpad * 8,
                      groups * 64u * A.dpad);
      }
      for (uint32_t kc = 0; kc < A.chunks; ++kc, ++g) {
        const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
        bool ready = true;
        if (lane == 0)
          ready = CL > 1 ? mbar_wait_cluster(smem_u32(&bar_empty[st]), ph ^ 1, &abort_flag, A.err, A.sleep_tma)
                         : mbar_wait(smem_u32(&bar_empty[st]), ph ^ 1, &abort_flag, A.err, A.sleep_tma);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { ok = false; break; }
        if (lane == 0) {
          const uint32_t full = smem_u32(&bar_full[st]);
          mbar_arrive_tx(full, TMA_B ? kStageBytes : kATile);
          tma_load_3d(sbase + st * kStageBytes, &pmap, (int)(kc * kBK), (int)(D.kt * kBM),
                      (int)(D.j * N + D.s), full);
          if (TMA_B && CL == 1)
            tma_load_3d(sbase + st * kStageBytes + kATile, &xmap, (int)(kc * kBK), (int)(D.qt * kBN),
                        (int)(D.j * A.s_count + D.sl), full);
          if (TMA_B && CL > 1)
            // rows [crank kBN / CL, ..) of the query tile, into every CTA of the cluster
            tma_load_3d_mc(sbase + st * kStageBytes + kATile + crank * (kBTile / CL), &xmap, (int)(kc * kBK),
                           (int)(D.qt * kBN + crank * (kBN / CL)), (int)(D.j * A.s_count + D.sl), full,
                           kMask);
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
    uint64_t g = 0;
    bool ok = true;
    for (uint32_t m = 0; ok; ++m) {
      Decoded D;
      if (!unit_of<CL>(m, A, D)) break;
      const uint32_t slot = m & 1, aph = (m >> 1) & 1;
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
          if (CL > 1) mma_commit_mc1(smem_u32(&bar_empty[st]), kMask);
          else mma_commit(smem_u32(&bar_empty[st]));
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma_commit(smem_u32(&bar_tfull[slot]));
      __syncwarp();
    }
  } else if (warp < kEpiWarp0) {
    if (TMA_B) {
      // the query-digit tiles arrive by TMA: nothing to produce
    } else {
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
    const uint32_t chunks = A.chunks;
    const uint32_t twoB = 2 * A.B;
    // this thread's item in dimension block 0 of the CTA's unit m (null past
    // the units or past 2B: such an item reads Y_b = 0x80.., all digits zero)
    auto unit_base = [&](uint32_t m) -> const ulonglong2* {
      Decoded D;
      if (!unit_of<CL>(m, A, D)) return nullptr;
      const uint32_t bc = D.qt * kQG + bcl;
      if (bc >= twoB) return nullptr;
      return reinterpret_cast<const ulonglong2*>(A.xm) +
             (((uint64_t)D.j * A.s_count + D.sl) * twoB + bc) * (A.dpad / 8) * 32 + il;
    };
    // dimension block k: 32 sixteen-byte words further; pair m at + 8 m
    auto load_item = [&](const ulonglong2* b0, uint32_t k, ulonglong2 (&dst)[4]) {
#pragma unroll
      for (int h = 0; h < 4; ++h)
        dst[h] = b0 ? __ldg(b0 + 32 * k + 8 * h) : make_ulonglong2(0x8080808080808080ull, 0x8080808080808080ull);
    };
    // Each warp fills its own 32 items (4 row groups x 8 dims) of every stage
    // and arrives on the stage's barrier itself, so warps run ahead of one
    // another; values are prefetched two chunks ahead.
    uint32_t fm = 0, fk = 0;
    const ulonglong2* fb = unit_base(fm);
    auto advance = [&]() {
      if (++fk == chunks) { fk = 0; ++fm; fb = unit_base(fm); }
    };
    ulonglong2 nx0[4], nx1[4];
    load_item(fb, fk, nx0);
    advance();
    load_item(fb, fk, nx1);
    advance();
    uint64_t g = 0;
    uint32_t cm = 0, ck = 0;
    Decoded Dc;
    bool have = unit_of<CL>(0, A, Dc);
    while (have) {
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
      store_digit_rows(base + st * kStageBytes + kATile, bcl, il, cur);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_full[st]));
      if (++ck == chunks) { ck = 0; ++cm; have = unit_of<CL>(cm, A, Dc); }
    }
    }
  } else {
    // ---------------- epilogue ----------------
    // Lane = database block k of the tile (see epilogue_values).  The first
    // slot of a pair is held in registers until the second one is done, then
    // both go out as one 16-byte word per output.
    const uint32_t quarter = warp & 3;            // TMEM lanes 32 quarter ..
    const uint32_t chalf = (warp - kEpiWarp0) >> 2;  // column half of the tile
    const uint32_t N = P.N, L = P.L;
    // the pair's first slot, [output i][epilogue thread] (conflict-free)
    uint64_t* held = reinterpret_cast<uint64_t*>(base + kStages * kStageBytes);
    const uint32_t et = threadIdx.x - 32 * kEpiWarp0;
    for (uint32_t m = 0; !abort_flag; ++m) {
      Decoded D;
      if (!unit_of<CL>(m, A, D)) break;
      const uint32_t slot = m & 1, aph = (m >> 1) & 1;
      // lane 0 waits for the accumulator, the warp follows its decision
      bool ready = true;
      if (lane == 0) ready = mbar_wait(smem_u32(&bar_tfull[slot]), aph, &abort_flag, A.err, A.sleep_epi);
      if (!__shfl_sync(0xffffffffu, (int)ready, 0)) break;
      tc_fence_after();
      const uint32_t k = D.kt * kBM + quarter * 32 + lane;
      const bool k_ok = k < A.K;
#pragma unroll
      for (uint32_t ci = 0; ci < 4; ++ci) {
        const uint32_t cc = chalf * 4 + ci;
        uint64_t res[4];
        epilogue_values(tmem + ((quarter * 32) << 16) + slot * kBN + cc * 32, A, P, D, res);
        if (slot == 0) {
#pragma unroll
          for (int o = 0; o < 4; ++o) held[(ci * 4 + o) * (32 * kEpiWarps) + et] = res[o];
        } else {
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            const uint32_t bc = D.qt * kQG + cc * 4 + o;
            if (k_ok && bc < 2 * A.B) {
              const uint32_t b = bc >> 1, c = bc & 1;
              uint64_t* dst = A.out + ((((uint64_t)b * A.K + k) * 2 + c) * L + D.j) * N + D.s - 1;
              const uint64_t h = held[(ci * 4 + o) * (32 * kEpiWarps) + et];
              if (A.out16) {
                *reinterpret_cast<ulonglong2*>(dst) = make_ulonglong2(h, res[o]);
              } else {
                dst[0] = h;
                dst[1] = res[o];
              }
            }
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
  if (CL > 1) cluster_barrier();  // no CTA leaves while a peer may still reach its memory
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// ------------------------------------------------------------------------
// The TMA-fed single-SM tile with whole-sector output stores.  The outputs of
// one unit (one slot) are 128 blocks x 32 (b, c) words, every one of them in
// a different 393 KB-apart row of the [B][K][2][L][N] response layout, so
// one slot alone can only write 8 bytes (or 16 for a slot pair) per row.
// Here a CTA takes four consecutive slots of the same (prime, database tile,
// query tile) back to back; the epilogue keeps the first two slots' results
// in registers and the third in shared memory, and writes each output row's
// four slots as one 32-byte store (a whole DRAM sector).  Both operands
// arrive by TMA, so the CTA has no producer warps: 10 warps (TMA, MMA, 8
// epilogue).  CL > 1: clusters that share each query tile by multicast, as in
// batched_mac_kernel.
// ------------------------------------------------------------------------
namespace quad {
constexpr int kEpiWarp0 = 2;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (kEpiWarp0 + kEpiWarps);  // 320
// stages + the third held slot (16 outputs per epilogue thread)
constexpr int kHeldBytes = 16 * 32 * kEpiWarps * 8;
constexpr int kSmem = kStages * kStageBytes + kHeldBytes + 1024;
}  // namespace quad

// Unit m of this CTA: quad p = cluster + (m / 4) (clusters in the grid) over
// A.units quads, decoded as ((j S/4 + s'/4) KTG + ktg) QT + qt; slot s' = 4
// (s'/4) + m % 4; database tile CL ktg + rank.
template <int CL>
__device__ __forceinline__ bool unit_of_quad(uint32_t m, const BatchArgs& A, Decoded& D) {
  const uint32_t cid = blockIdx.x / CL, rank = blockIdx.x % CL, ncl = gridDim.x / CL;
  const uint64_t p = cid + (uint64_t)(m >> 2) * ncl;
  if (p >= A.units) return false;
  const uint32_t quarter = A.s_count >> 2;
  const uint32_t ktg = A.KT / CL;
  uint32_t r = (uint32_t)p;
  D.qt = r % A.QT;
  r /= A.QT;
  D.kt = (r % ktg) * CL + rank;
  r /= ktg;
  D.sl = 4 * (r % quarter) + (m & 3);
  D.s = A.s_begin + D.sl;
  D.j = r / quarter;
  return true;
}

__device__ __forceinline__ void st_global_v4_b64(uint64_t* p, uint64_t a, uint64_t b, uint64_t c,
                                                 uint64_t d) {
  asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d)
               : "memory");
}

template <int CL>
__global__ void __launch_bounds__(quad::kThreads, 1)
batched_mac_quad_kernel(const __grid_constant__ CUtensorMap pmap, const __grid_constant__ CUtensorMap xmap,
                        PrimeSet P, BatchArgs A) {
  constexpr int kEpiWarp0 = quad::kEpiWarp0;
  constexpr int kEpiWarps = quad::kEpiWarps;
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
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), CL);
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
  if (CL > 1) cluster_barrier();  // every CTA's barriers exist before any multicast
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;
  const uint32_t N = P.N;
  const uint32_t crank = blockIdx.x % CL;
  constexpr uint16_t kMask = (uint16_t)((1u << CL) - 1);

  if (warp == 0) {
    // ---------------- TMA producer: database tile + query tile ----------------
    uint64_t g = 0;
    bool ok = true;
    for (uint32_t m = 0; ok; ++m) {
      Decoded D;
      if (!unit_of_quad<CL>(m, A, D)) break;
      for (uint32_t kc = 0; kc < A.chunks; ++kc, ++g) {
        const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
        bool ready = true;
        if (lane == 0)
          ready = CL > 1 ? mbar_wait_cluster(smem_u32(&bar_empty[st]), ph ^ 1, &abort_flag, A.err, A.sleep_tma)
                         : mbar_wait(smem_u32(&bar_empty[st]), ph ^ 1, &abort_flag, A.err, A.sleep_tma);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { ok = false; break; }
        if (lane == 0) {
          const uint32_t full = smem_u32(&bar_full[st]);
          mbar_arrive_tx(full, kStageBytes);
          tma_load_3d(sbase + st * kStageBytes, &pmap, (int)(kc * kBK), (int)(D.kt * kBM),
                      (int)(D.j * N + D.s), full);
          if (CL == 1)
            tma_load_3d(sbase + st * kStageBytes + kATile, &xmap, (int)(kc * kBK), (int)(D.qt * kBN),
                        (int)(D.j * A.s_count + D.sl), full);
          else
            tma_load_3d_mc(sbase + st * kStageBytes + kATile + crank * (kBTile / CL), &xmap, (int)(kc * kBK),
                           (int)(D.qt * kBN + crank * (kBN / CL)), (int)(D.j * A.s_count + D.sl), full,
                           kMask);
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
    uint64_t g = 0;
    bool ok = true;
    for (uint32_t m = 0; ok; ++m) {
      Decoded D;
      if (!unit_of_quad<CL>(m, A, D)) break;
      const uint32_t slot = m & 1, aph = (m >> 1) & 1;
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
          if (CL > 1) mma_commit_mc1(smem_u32(&bar_empty[st]), kMask);
          else mma_commit(smem_u32(&bar_empty[st]));
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma_commit(smem_u32(&bar_tfull[slot]));
      __syncwarp();
    }
  } else {
    // ---------------- epilogue ----------------
    // Lane = database block k of the tile; each thread owns 16 outputs (4
    // column chunks x 4 (b, c) rows) of its block per slot.  Slots 0..2 of a
    // quad are held in registers, slot 3 writes all four.
    const uint32_t quarter = warp & 3;                 // TMEM lanes 32 quarter ..
    const uint32_t chalf = (warp - kEpiWarp0) >> 2;    // column half of the tile
    const uint32_t L = P.L;
    const uint32_t et = threadIdx.x - 32 * kEpiWarp0;
    // slots 0, 1 of a quad in registers; slot 2 in shared memory, [output
    // i][epilogue thread] (conflict-free)
    uint64_t held[2][16];
    uint64_t* held2 = reinterpret_cast<uint64_t*>(base + kStages * kStageBytes);
    bool live = true;
    for (uint32_t m = 0; live && !abort_flag; m += 4) {
#pragma unroll
      for (int sub = 0; sub < 4; ++sub) {
        Decoded D;
        if (!live || !unit_of_quad<CL>(m + sub, A, D)) { live = false; break; }
        const uint32_t u = m + sub;
        const uint32_t slot = u & 1, aph = (u >> 1) & 1;
        bool ready = true;
        if (lane == 0) ready = mbar_wait(smem_u32(&bar_tfull[slot]), aph, &abort_flag, A.err, A.sleep_epi);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { live = false; break; }
        tc_fence_after();
        const uint32_t k = D.kt * kBM + quarter * 32 + lane;
        const bool k_ok = k < A.K;
#pragma unroll
        for (uint32_t ci = 0; ci < 4; ++ci) {
          const uint32_t cc = chalf * 4 + ci;
          uint64_t res[4];
          epilogue_values(tmem + ((quarter * 32) << 16) + slot * kBN + cc * 32, A, P, D, res);
          if (sub < 2) {
#pragma unroll
            for (int o = 0; o < 4; ++o) held[sub][ci * 4 + o] = res[o];
          } else if (sub == 2) {
#pragma unroll
            for (int o = 0; o < 4; ++o) held2[(ci * 4 + o) * (32 * kEpiWarps) + et] = res[o];
          } else {
#pragma unroll
            for (int o = 0; o < 4; ++o) {
              const uint32_t bc = D.qt * kQG + cc * 4 + o;
              if (k_ok && bc < 2 * A.B) {
                const uint32_t b = bc >> 1, c = bc & 1;
                uint64_t* dst = A.out + ((((uint64_t)b * A.K + k) * 2 + c) * L + D.j) * N + D.s - 3;
                const uint64_t h2 = held2[(ci * 4 + o) * (32 * kEpiWarps) + et];
                if (A.out16 == 2) {
                  st_global_v4_b64(dst, held[0][ci * 4 + o], held[1][ci * 4 + o], h2, res[o]);
                } else {
                  dst[0] = held[0][ci * 4 + o];
                  dst[1] = held[1][ci * 4 + o];
                  dst[2] = h2;
                  dst[3] = res[o];
                }
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_tempty[slot]));
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (CL > 1) cluster_barrier();  // no CTA leaves while a peer may still reach its memory
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// ------------------------------------------------------------------------
// The same contraction on CTA pairs (cluster of 2, tcgen05 cta_group::2): one
// MMA of M = 256 (128 database blocks from each CTA's shared memory) by
// N = 256 query rows (128 generated by each CTA) by K = 16.  Per SM this
// halves the query-digit rows the producers write and the B operand the MMA
// reads from shared memory, the resource the single-CTA tile is bound by.
// The even CTA (rank 0) issues the MMAs and owns the stage-full and
// accumulator-empty barriers; the odd CTA's TMA completes its bytes on them,
// its producers and epilogue arrive remotely, and the MMA completion is
// multicast to the stage-empty and accumulator-full barriers of both.
// ------------------------------------------------------------------------
namespace pair {
constexpr int kStages = 6;
constexpr int kXStages = 4;               // query-multiple tiles in flight (TMA)
constexpr int kBM = 128;                  // database blocks per CTA (M = 256 per pair)
constexpr int kBN = 256;                  // query rows per pair (N)
constexpr int kBNh = 128;                 // query rows generated per CTA
constexpr int kBK = 64;
constexpr int kQG = kBN / 8;              // (b, c) row groups per pair tile
constexpr int kQGh = kBNh / 8;            // per CTA
constexpr int kATile = kBM * kBK * 2;     // 16 KB
constexpr int kBTile = kBNh * kBK * 2;    // 16 KB
constexpr int kStageBytes = kATile + kBTile;
constexpr int kXTile = kQGh * 8 * 64;     // 16 row groups x 8 dimensions x 64 bytes = 8 KB
constexpr int kSmem = kStages * kStageBytes + kXStages * kXTile + 1024;
constexpr int kProdWarp0 = 2;
constexpr int kProdWarps = 4;
static_assert(32 * kProdWarps == kQGh * 8, "one (row group, dimension) item per producer thread");
constexpr int kEpiWarp0 = kProdWarp0 + kProdWarps;    // 6
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (kEpiWarp0 + kEpiWarps);  // 448
// kind::f16: D fp32, A and B fp16, both K-major, M = 256, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}  // namespace pair

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// shared::cluster address of the same variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait (cluster-scope acquire), as mbar_wait.
__device__ __forceinline__ bool mbar_wait_cl(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                             int* err, uint32_t sleep_ns = 0) {
  const unsigned long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_cluster(bar, parity)) return true;
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

// Tile load into this CTA's shared memory whose completion is counted on an
// mbarrier of either CTA of the pair (cluster address).
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map, int x, int y,
                                                 int z, uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar_cluster)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            int w, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mma_f16_pair(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                             uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(pair::kIdesc), "r"(accumulate));
}

// completion of this thread's prior MMAs arrives on the barrier at the same
// offset in every CTA of `mask`
__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar), "h"(mask)
      : "memory");
}

// TMA_B: each CTA's half of the query-digit tile arrives by TMA from the fp16
// rows of expand_query_f16_kernel (xmap, boxes of 128 rows) and the producer
// warps stay idle; otherwise xmap holds the byte-interleaved multiples and the
// producers generate the digits.
template <bool TMA_B>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(pair::kThreads, 1)
batched_mac_pair_kernel(const __grid_constant__ CUtensorMap pmap, const __grid_constant__ CUtensorMap xmap,
                        PrimeSet P, BatchArgs A) {
  constexpr int kStages = pair::kStages;
  constexpr int kXStages = pair::kXStages;
  constexpr int kXTile = pair::kXTile;
  constexpr int kBM = pair::kBM;
  constexpr int kBN = pair::kBN;
  constexpr int kBK = pair::kBK;
  constexpr int kQG = pair::kQG;
  constexpr int kQGh = pair::kQGh;
  constexpr int kATile = pair::kATile;
  constexpr int kStageBytes = pair::kStageBytes;
  constexpr int kProdWarp0 = pair::kProdWarp0;
  constexpr int kProdWarps = pair::kProdWarps;
  constexpr int kEpiWarp0 = pair::kEpiWarp0;
  constexpr int kEpiWarps = pair::kEpiWarps;
  extern __shared__ __align__(1024) uint8_t dsmem[];
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages];
  __shared__ __align__(8) uint64_t bar_tfull[2], bar_tempty[2], bar_done;
  __shared__ __align__(8) uint64_t bar_xfull[kXStages], bar_xempty[kXStages];
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;

  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const uint32_t cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  uint8_t* base = dsmem + ((1024 - (smem_u32(dsmem) & 1023)) & 1023);
  const uint32_t sbase = smem_u32(base);
  const uint32_t xbase = sbase + kStages * kStageBytes;  // query-multiple tiles

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kXStages; ++s) {
      mbar_init(smem_u32(&bar_xfull[s]), 1);
      mbar_init(smem_u32(&bar_xempty[s]), kProdWarps);
    }
    for (int s = 0; s < kStages; ++s) {
      // leader: its TMA thread (expecting both CTAs' bytes) + both CTAs' producers
      mbar_init(smem_u32(&bar_full[s]), TMA_B ? 1 : 1 + 2 * kProdWarps);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bar_tfull[a]), 1);
      mbar_init(smem_u32(&bar_tempty[a]), 2 * kEpiWarps);
    }
    mbar_init(smem_u32(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    // one warp of each CTA allocates the same columns in both
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&tmem_base_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // barriers of both CTAs initialised before any remote arrival
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;
  const uint32_t N = P.N;

  if (warp == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    uint64_t g = 0;
    bool ok = true;
    for (uint64_t u = cl; u < A.units && ok; u += ncl) {
      const Decoded D = decode_unit((uint32_t)u, P.logN, A);
      const uint64_t pu = u + (uint64_t)A.prefetch_units * ncl;
      if (lane == 0 && A.prefetch_units && pu < A.units) {
        const Decoded F = decode_unit((uint32_t)pu, P.logN, A);
        const uint32_t r0 = F.kt * 2 * kBM + rank * kBM;
        if (r0 < A.K) {
          const uint32_t rows = A.K - r0 < (uint32_t)kBM ? A.K - r0 : (uint32_t)kBM;
          prefetch_l2(A.plimb + (((uint64_t)F.j * N + F.s) * A.K + r0) * 8 * A.dpad,
                      rows * 16u * A.dpad);
        }
        const uint32_t twoB = 2 * A.B, bc0 = F.qt * kQG + rank * kQGh;
        if (bc0 < twoB) {
          const uint32_t groups = twoB - bc0 < (uint32_t)kQGh ? twoB - bc0 : (uint32_t)kQGh;
          if (TMA_B)
            prefetch_l2(A.xh + (((uint64_t)F.j * A.s_count + F.sl) * 8 * twoB + 8 * bc0) * 8 * A.dpad,
                        groups * 128u * A.dpad);
          else
            prefetch_l2(A.xm + (((uint64_t)F.j * A.s_count + F.sl) * twoB + bc0) * A.dpad * 8,
                        groups * 64u * A.dpad);
        }
      }
      for (uint32_t kc = 0; kc < A.chunks; ++kc, ++g) {
        const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
        const uint32_t xs = (uint32_t)(g % kXStages), xph = (uint32_t)((g / kXStages) & 1);
        bool ready = true;
        if (!TMA_B) {
          // this CTA's query multiples of the stage: 16 row groups x 8 dimensions
          if (lane == 0) ready = mbar_wait_cl(smem_u32(&bar_xempty[xs]), xph ^ 1, &abort_flag, A.err, A.sleep_tma);
          if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { ok = false; break; }
          if (lane == 0) {
            const uint32_t xf = smem_u32(&bar_xfull[xs]);
            mbar_arrive_tx(xf, kXTile);
            tma_load_4d(xbase + xs * kXTile, &xmap, 0, (int)kc, (int)(D.qt * kQG + rank * kQGh),
                        (int)(D.j * A.s_count + D.sl), xf);
          }
          __syncwarp();
        }
        if (lane == 0) ready = mbar_wait_cl(smem_u32(&bar_empty[st]), ph ^ 1, &abort_flag, A.err, A.sleep_tma);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { ok = false; break; }
        if (lane == 0) {
          const uint32_t full = smem_u32(&bar_full[st]);
          if (rank == 0) mbar_arrive_tx(full, TMA_B ? 2 * kStageBytes : 2 * kATile);
          tma_load_3d_pair(sbase + st * kStageBytes, &pmap, (int)(kc * kBK),
                           (int)(D.kt * 2 * kBM + rank * kBM), (int)(D.j * N + D.s),
                           map_rank(full, 0));
          if (TMA_B)
            tma_load_3d_pair(sbase + st * kStageBytes + kATile, &xmap, (int)(kc * kBK),
                             (int)(D.qt * kBN + rank * pair::kBNh), (int)(D.j * A.s_count + D.sl),
                             map_rank(full, 0));
        }
        __syncwarp();
      }
    }
    if (!ok && lane == 0) {
      // copies in flight complete on the leader's barriers: give them a
      // bounded moment before the CTA may leave
      const unsigned long long t0 = clock64();
      while (clock64() - t0 < (1ull << 22)) {
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer (rank 0 only) ----------------
    if (rank == 0) {
      uint64_t g = 0, r = 0;
      bool ok = true;
      for (uint64_t u = cl; u < A.units && ok; u += ncl, ++r) {
        const uint32_t slot = (uint32_t)(r & 1), aph = (uint32_t)((r >> 1) & 1);
        bool ready = true;
        if (lane == 0) ready = mbar_wait_cl(smem_u32(&bar_tempty[slot]), aph ^ 1, &abort_flag, A.err, A.sleep_mma);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) break;
        tc_fence_after();
        const uint32_t dt = tmem + slot * kBN;
        for (uint32_t kc = 0; kc < A.chunks; ++kc, ++g) {
          const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
          if (lane == 0) ready = mbar_wait_cl(smem_u32(&bar_full[st]), ph, &abort_flag, A.err, A.sleep_mma);
          if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { ok = false; break; }
          tc_fence_after();
          if (lane == 0) {
            const uint32_t a_addr = sbase + st * kStageBytes, b_addr = a_addr + kATile;
            const uint64_t ad = smem_desc(a_addr), bd = smem_desc(b_addr);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
              mma_f16_pair(dt, ad + 2 * k, bd + 2 * k, (kc > 0 || k > 0) ? 1u : 0u);
            mma_commit_mc(smem_u32(&bar_empty[st]), 0x3);
          }
          __syncwarp();
        }
        if (!ok) break;
        if (lane == 0) mma_commit_mc(smem_u32(&bar_tfull[slot]), 0x3);
        __syncwarp();
      }
      // every MMA issued has completed before the pair may tear down
      if (lane == 0) {
        mma_commit_mc(smem_u32(&bar_done), 0x1);
        const unsigned long long t0 = clock64();
        while (!mbar_try_cluster(smem_u32(&bar_done), 0) && clock64() - t0 < kWaitCycles) {
        }
      }
      __syncwarp();
    }
  } else if (warp < kEpiWarp0) {
    if (TMA_B) {
      // the query-digit halves arrive by TMA: nothing to produce
    } else {
    // ---------------- query-digit producers (both CTAs) ----------------
    // this CTA's half of the tile's query rows: row groups rank 16 .. rank 16
    // + 15; their multiples arrive by TMA (rows past 2B read as zero, whose
    // digit columns are never stored)
    const uint32_t pt = threadIdx.x - 32 * kProdWarp0;
    const uint32_t bcl = pt >> 3, il = pt & 7;
    const uint32_t units = (uint32_t)A.units, chunks = A.chunks;
    uint64_t g = 0;
    for (uint32_t cu = cl; cu < units; cu += ncl) {
      bool ok = true;
      for (uint32_t kc = 0; kc < chunks; ++kc, ++g) {
        const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
        const uint32_t xs = (uint32_t)(g % kXStages), xph = (uint32_t)((g / kXStages) & 1);
        bool ready = true;
        if (lane == 0) ready = mbar_wait_cl(smem_u32(&bar_xfull[xs]), xph, &abort_flag, A.err, A.sleep_prod);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { ok = false; break; }
        // item (bcl, il): pair m at 16-byte word 32 bcl + 8 m + il (conflict-free)
        const ulonglong2* xt = reinterpret_cast<const ulonglong2*>(base + kStages * kStageBytes + xs * kXTile);
        ulonglong2 cur[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) cur[m] = xt[32 * bcl + 8 * m + il];
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_xempty[xs]));
        if (lane == 0) ready = mbar_wait_cl(smem_u32(&bar_empty[st]), ph ^ 1, &abort_flag, A.err, A.sleep_prod);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { ok = false; break; }
        store_digit_rows(base + st * kStageBytes + kATile, bcl, il, cur);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(map_rank(smem_u32(&bar_full[st]), 0));
      }
      if (!ok) break;
    }
    }
  } else {
    // ---------------- epilogue (both CTAs) ----------------
    // Lane = database block k (this CTA's 128 of the pair's 256); all 256
    // query columns of the pair tile.
    const uint32_t quarter = warp & 3;
    const uint32_t chalf = (warp - kEpiWarp0) >> 2;
    uint64_t r = 0;
    for (uint64_t u = cl; u < A.units && !abort_flag; u += ncl, ++r) {
      const uint32_t slot = (uint32_t)(r & 1), aph = (uint32_t)((r >> 1) & 1);
      bool ready = true;
      if (lane == 0) ready = mbar_wait_cl(smem_u32(&bar_tfull[slot]), aph, &abort_flag, A.err, A.sleep_epi);
      if (!__shfl_sync(0xffffffffu, (int)ready, 0)) break;
      tc_fence_after();
      const Decoded D = decode_unit((uint32_t)u, P.logN, A);
      const uint32_t k = D.kt * 2 * kBM + rank * kBM + quarter * 32 + lane;
      for (uint32_t cc = chalf * (kBN / 64); cc < (chalf + 1) * (kBN / 64); ++cc)
        epilogue_chunk(tmem + ((quarter * 32) << 16) + slot * kBN + cc * 32, A, P, D, k, k < A.K,
                       D.qt * kQG + cc * 4);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(map_rank(smem_u32(&bar_tempty[slot]), 0));
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // no CTA leaves while its peer may still reach its memory
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// ------------------------------------------------------------------------
// Tile 8: the four-slot epilogue on CTA pairs.  One tcgen05 MMA of M = 256
// (128 database blocks in each CTA) by N = 256 query rows (128 held by each
// CTA) by K = 16; both operands arrive by TMA.  A stage is 32 KB per CTA
// instead of the single-SM tile's 48 KB for the same MMA work per SM, so six
// stages fit beside the epilogue's held slot: half again as much work in
// flight to cover the load latency and the stage hand-off, and a third less
// traffic from L2 and into shared memory per product.
// Roles as in batched_mac_quad_kernel; the even CTA's MMA thread issues for
// both, its stage-full barrier counts both CTAs' bytes, and the MMA
// completions are multicast to the stage-empty and accumulator-full barriers
// of both CTAs.  Each CTA's epilogue reads its own 128 TMEM lanes and arrives
// on the even CTA's accumulator-empty barrier.
// ------------------------------------------------------------------------
namespace pq {
constexpr int kStages = 6;
constexpr int kBM = 128;                  // database blocks per CTA (M = 256 per pair)
constexpr int kBN = 256;                  // query rows per pair tile (N)
constexpr int kBNh = 128;                 // query rows held per CTA
constexpr int kATile = kBM * kBK * 2;     // 16 KB
constexpr int kBTile = kBNh * kBK * 2;    // 16 KB
constexpr int kStageBytes = kATile + kBTile;
constexpr int kEpiWarp0 = 2;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (kEpiWarp0 + kEpiWarps);  // 320
constexpr int kHeldBytes = 16 * 32 * kEpiWarps * 8;
constexpr int kSmem = kStages * kStageBytes + kHeldBytes + 1024;
static_assert(kSmem <= 227 * 1024, "stages + held slot fit one CTA's shared memory");
}  // namespace pq

// Unit m of this pair: quad p = pair + (m / 4) (pairs in the grid) over
// A.units quads, decoded as ((j S/4 + s'/4) KT + kt) QT + qt with kt a
// 256-block pair tile; slot s' = 4 (s'/4) + m % 4.  Both CTAs decode the same
// unit; rank r takes blocks 256 kt + 128 r .. + 127.
__device__ __forceinline__ bool unit_of_pq(uint32_t m, const BatchArgs& A, Decoded& D) {
  const uint32_t cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const uint64_t p = cid + (uint64_t)(m >> 2) * ncl;
  if (p >= A.units) return false;
  const uint32_t quarter = A.s_count >> 2;
  uint32_t r = (uint32_t)p;
  D.qt = r % A.QT;
  r /= A.QT;
  D.kt = r % A.KT;
  r /= A.KT;
  D.sl = 4 * (r % quarter) + (m & 3);
  D.s = A.s_begin + D.sl;
  D.j = r / quarter;
  return true;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(pq::kThreads, 1)
batched_mac_pairq_kernel(const __grid_constant__ CUtensorMap pmap, const __grid_constant__ CUtensorMap xmap,
                         PrimeSet P, BatchArgs A) {
  constexpr int kStages = pq::kStages;
  constexpr int kEpiWarp0 = pq::kEpiWarp0;
  constexpr int kEpiWarps = pq::kEpiWarps;
  constexpr int kStageBytes = pq::kStageBytes;
  extern __shared__ __align__(1024) uint8_t dsmem[];
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages];
  __shared__ __align__(8) uint64_t bar_tfull[2], bar_tempty[2], bar_done;
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;

  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  uint8_t* base = dsmem + ((1024 - (smem_u32(dsmem) & 1023)) & 1023);
  const uint32_t sbase = smem_u32(base);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);    // even CTA: its TMA thread, both CTAs' bytes
      mbar_init(smem_u32(&bar_empty[s]), 1);   // the even CTA's multicast commit
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bar_tfull[a]), 1);
      mbar_init(smem_u32(&bar_tempty[a]), 2 * kEpiWarps);
    }
    mbar_init(smem_u32(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&tmem_base_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // barriers of both CTAs initialised before any remote arrival
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;
  const uint32_t N = P.N;

  if (warp == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    uint64_t g = 0;
    bool ok = true;
    for (uint32_t m = 0; ok; ++m) {
      Decoded D;
      if (!unit_of_pq(m, A, D)) break;
      for (uint32_t kc = 0; kc < A.chunks; ++kc, ++g) {
        const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
        bool ready = true;
        if (lane == 0) ready = mbar_wait_cl(smem_u32(&bar_empty[st]), ph ^ 1, &abort_flag, A.err, A.sleep_tma);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { ok = false; break; }
        if (lane == 0) {
          const uint32_t full = smem_u32(&bar_full[st]);
          if (rank == 0) mbar_arrive_tx(full, 2 * kStageBytes);
          const uint32_t full0 = map_rank(full, 0);
          tma_load_3d_pair(sbase + st * kStageBytes, &pmap, (int)(kc * kBK),
                           (int)(D.kt * 2 * pq::kBM + rank * pq::kBM), (int)(D.j * N + D.s), full0);
          tma_load_3d_pair(sbase + st * kStageBytes + pq::kATile, &xmap, (int)(kc * kBK),
                           (int)(D.qt * pq::kBN + rank * pq::kBNh), (int)(D.j * A.s_count + D.sl), full0);
        }
        __syncwarp();
      }
    }
    if (!ok && lane == 0) {
      // copies in flight complete on the even CTA's barriers: give them a
      // bounded moment before the CTA may leave
      const unsigned long long t0 = clock64();
      while (clock64() - t0 < (1ull << 22)) {
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer (even CTA) ----------------
    if (rank == 0) {
      uint64_t g = 0;
      bool ok = true;
      for (uint32_t m = 0; ok; ++m) {
        Decoded D;
        if (!unit_of_pq(m, A, D)) break;
        const uint32_t slot = m & 1, aph = (m >> 1) & 1;
        bool ready = true;
        if (lane == 0) ready = mbar_wait_cl(smem_u32(&bar_tempty[slot]), aph ^ 1, &abort_flag, A.err, A.sleep_mma);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) break;
        tc_fence_after();
        const uint32_t dt = tmem + slot * pq::kBN;
        for (uint32_t kc = 0; kc < A.chunks; ++kc, ++g) {
          const uint32_t st = (uint32_t)(g % kStages), ph = (uint32_t)((g / kStages) & 1);
          if (lane == 0) ready = mbar_wait_cl(smem_u32(&bar_full[st]), ph, &abort_flag, A.err, A.sleep_mma);
          if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { ok = false; break; }
          tc_fence_after();
          if (lane == 0) {
            const uint32_t a_addr = sbase + st * kStageBytes, b_addr = a_addr + pq::kATile;
            const uint64_t ad = smem_desc(a_addr), bd = smem_desc(b_addr);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
              mma_f16_pair(dt, ad + 2 * k, bd + 2 * k, (kc > 0 || k > 0) ? 1u : 0u);
            mma_commit_mc(smem_u32(&bar_empty[st]), 0x3);
          }
          __syncwarp();
        }
        if (!ok) break;
        if (lane == 0) mma_commit_mc(smem_u32(&bar_tfull[slot]), 0x3);
        __syncwarp();
      }
      // every MMA issued has completed before the pair may tear down
      if (lane == 0) {
        mma_commit_mc(smem_u32(&bar_done), 0x1);
        const unsigned long long t0 = clock64();
        while (!mbar_try_cluster(smem_u32(&bar_done), 0) && clock64() - t0 < kWaitCycles) {
        }
      }
      __syncwarp();
    }
  } else {
    // ---------------- epilogue (both CTAs) ----------------
    // Lane = database block of this CTA's 128; each thread owns 16 outputs
    // (4 column chunks x 4 (b, c) rows) per slot.  Slots 0, 1 of a quad are
    // held in registers, slot 2 in shared memory, slot 3 writes all four as
    // one 32-byte store per output.
    const uint32_t quarter = warp & 3;
    const uint32_t chalf = (warp - kEpiWarp0) >> 2;
    const uint32_t L = P.L;
    const uint32_t et = threadIdx.x - 32 * kEpiWarp0;
    uint64_t held[2][16];
    uint64_t* held2 = reinterpret_cast<uint64_t*>(base + kStages * kStageBytes);
    bool live = true;
    for (uint32_t m = 0; live && !abort_flag; m += 4) {
#pragma unroll
      for (int sub = 0; sub < 4; ++sub) {
        Decoded D;
        if (!live || !unit_of_pq(m + sub, A, D)) { live = false; break; }
        const uint32_t u = m + sub;
        const uint32_t slot = u & 1, aph = (u >> 1) & 1;
        bool ready = true;
        if (lane == 0) ready = mbar_wait_cl(smem_u32(&bar_tfull[slot]), aph, &abort_flag, A.err, A.sleep_epi);
        if (!__shfl_sync(0xffffffffu, (int)ready, 0)) { live = false; break; }
        tc_fence_after();
        const uint32_t k = D.kt * 2 * pq::kBM + rank * pq::kBM + quarter * 32 + lane;
        const bool k_ok = k < A.K;
#pragma unroll
        for (uint32_t ci = 0; ci < 4; ++ci) {
          const uint32_t cc = chalf * 4 + ci;
          uint64_t res[4];
          epilogue_values(tmem + ((quarter * 32) << 16) + slot * pq::kBN + cc * 32, A, P, D, res);
          if (sub < 2) {
#pragma unroll
            for (int o = 0; o < 4; ++o) held[sub][ci * 4 + o] = res[o];
          } else if (sub == 2) {
#pragma unroll
            for (int o = 0; o < 4; ++o) held2[(ci * 4 + o) * (32 * kEpiWarps) + et] = res[o];
          } else {
#pragma unroll
            for (int o = 0; o < 4; ++o) {
              const uint32_t bc = D.qt * kQG + cc * 4 + o;
              if (k_ok && bc < 2 * A.B) {
                const uint32_t b = bc >> 1, c = bc & 1;
                uint64_t* dst = A.out + ((((uint64_t)b * A.K + k) * 2 + c) * L + D.j) * N + D.s - 3;
                const uint64_t h2 = held2[(ci * 4 + o) * (32 * kEpiWarps) + et];
                if (A.out16 == 2) {
                  st_global_v4_b64(dst, held[0][ci * 4 + o], held[1][ci * 4 + o], h2, res[o]);
                } else {
                  dst[0] = held[0][ci * 4 + o];
                  dst[1] = held[1][ci * 4 + o];
                  dst[2] = h2;
                  dst[3] = res[o];
                }
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(map_rank(smem_u32(&bar_tempty[slot]), 0));
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // no CTA leaves while its peer may still reach its memory
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem));
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
    tile[e] = i < d ? join30(pt[(((uint64_t)k * L + j) * d + i) * N + s0 + s]) : 0;
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

// 256^b mod q_j and Shoup companions, passed by value (no host buffer to copy,
// so a launch can be captured into a CUDA graph)
struct W256 {
  uint64_t w[kMaxPrimes][8];
  uint64_t ws[kMaxPrimes][8];
};

// X_b = ct 256^b mod q for b = 0..7, for the slots [s_begin, s_begin + S),
// stored for the digit producers as Y_b = X_b + 0x8080808080808080 (whose
// bytes are the balanced base-256 digits plus 128; no carry out, X_b < 2^62)
// with the bytes of Y_2m and Y_2m+1 interleaved into one 16-byte word Z_m.
// Layout, in 16-byte words: xm[j][s'][bc][i / 8][m][i % 8], bc = 2 b_query + c,
// i < dpad (dimensions d .. dpad - 1 hold Y_b = 0x80.., all digits zero).  A
// block takes (j, bc, 8 dimensions, 32 slots): coalesced ciphertext reads
// along the slots, a shared-memory transpose, then 512 contiguous bytes per
// slot.
__global__ void __launch_bounds__(256) expand_query_kernel(PrimeSet P, const uint64_t* __restrict__ ct,
                                    uint32_t B, uint32_t d, uint32_t dpad, uint32_t s_begin, uint32_t S,
                                    const W256 W,
                                    ulonglong2* __restrict__ xm) {
  __shared__ ulonglong2 tile[32][4][8];  // [slot][m][dim in block]
  const uint32_t s0 = blockIdx.x * 32, ib = blockIdx.y;
  const uint32_t j = blockIdx.z / (2 * B), bc = blockIdx.z % (2 * B);
  const uint32_t b = bc >> 1, c = bc & 1;
  const uint32_t N = P.N, L = P.L;
  const uint64_t q = P.q[j];
  {
    const uint32_t il = threadIdx.x >> 5, sl = threadIdx.x & 31;
    const uint32_t i = ib * 8 + il;
    uint64_t v[8];
    if (i < d && s0 + sl < S) {
      const uint64_t X = ct[((((uint64_t)b * d + i) * 2 + c) * L + j) * N + s_begin + s0 + sl];
      v[0] = X;
#pragma unroll
      for (int k = 1; k < 8; ++k) v[k] = mul_shoup(X, W.w[j][k], W.ws[j][k], q);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = 0;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const uint64_t y0 = v[2 * m] + 0x8080808080808080ull, y1 = v[2 * m + 1] + 0x8080808080808080ull;
      const uint32_t l0 = (uint32_t)y0, h0 = (uint32_t)(y0 >> 32), l1 = (uint32_t)y1, h1 = (uint32_t)(y1 >> 32);
      const uint64_t zx = (uint64_t)__byte_perm(l0, l1, 0x5140) | ((uint64_t)__byte_perm(l0, l1, 0x7362) << 32);
      const uint64_t zy = (uint64_t)__byte_perm(h0, h1, 0x5140) | ((uint64_t)__byte_perm(h0, h1, 0x7362) << 32);
      tile[sl][m][il] = make_ulonglong2(zx, zy);
    }
  }
  __syncthreads();
  // warp w writes slots w, w + 8, ..: 32 words = the slot's 512-byte block
  const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint32_t sl = w; sl < 32; sl += 8) {
    if (s0 + sl >= S) break;
    xm[((((uint64_t)j * S + s0 + sl) * 2 * B + bc) * (dpad / 8) + ib) * 32 + lane] =
        tile[sl][lane >> 3][lane & 7];
  }
}

// The query-digit rows of the TMA-fed tiles, fp16, for the slots [s_begin,
// s_begin + S): xh[j][s'][8 bc + a][8 i + b] = digit a of X_b = ct[bc][i]
// 256^b mod q_j (balanced base-256 digits in [-128, 127]: the bytes of X_b +
// 0x80..80, minus 128), zero for i >= d; bc = 2 b_query + c.  This is the
// B operand of the contraction exactly as the MMA reads it (rows (bc, a),
// contraction (i, b)), so the MAC kernel moves it with plain tile copies.
// A block takes 4 consecutive slots of one prime, whose rows are 4
// contiguous 16 B x 8 dpad x 2-byte regions, and writes them whole: a thread
// takes (bc, i) items (i fastest) and reads the item's 4 slots as one 32-byte
// sector; a warp then stores 512 contiguous bytes per (slot, digit row).
__global__ void __launch_bounds__(256) expand_query_f16_kernel(PrimeSet P, const uint64_t* __restrict__ ct,
                                    uint32_t B, uint32_t d, uint32_t dpad, uint32_t s_begin, uint32_t S,
                                    const W256 W, uint4* __restrict__ xh) {
  const uint32_t s0 = blockIdx.x * 4, j = blockIdx.y;
  const uint32_t N = P.N, L = P.L;
  const uint64_t q = P.q[j];
  const uint32_t ns = S - s0 < 4 ? S - s0 : 4;        // slots of this block in the range
  const uint32_t items = 2 * B * dpad;
  for (uint32_t it = threadIdx.x; it < items; it += blockDim.x) {
    const uint32_t i = it % dpad, bc = it / dpad;
    const uint32_t b = bc >> 1, c = bc & 1;
    uint64_t x[4] = {0, 0, 0, 0};
    if (i < d) {
      const uint64_t* src = ct + ((((uint64_t)b * d + i) * 2 + c) * L + j) * N + s_begin + s0;
      if (ns == 4 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
        const ulonglong2 u0 = __ldcs(reinterpret_cast<const ulonglong2*>(src));
        const ulonglong2 u1 = __ldcs(reinterpret_cast<const ulonglong2*>(src) + 1);
        x[0] = u0.x;
        x[1] = u0.y;
        x[2] = u1.x;
        x[3] = u1.y;
      } else {
        for (uint32_t sl = 0; sl < ns; ++sl) x[sl] = src[sl];
      }
    }
#pragma unroll
    for (uint32_t sl = 0; sl < 4; ++sl) {
      if (sl >= ns) break;
      uint64_t v[8];
      v[0] = x[sl];
#pragma unroll
      for (int k = 1; k < 8; ++k) v[k] = mul_shoup(x[sl], W.w[j][k], W.ws[j][k], q);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] += 0x8080808080808080ull;  // bytes = digits + 128
      uint4* row = xh + (((uint64_t)j * S + s0 + sl) * 16 * B + 8 * bc) * dpad + i;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        uint32_t h[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          // fp16 of (byte - 128) for b = 2m, 2m + 1: 0x64vv = 1024 + v exactly,
          // minus 1152
          const uint32_t lo = (uint32_t)(v[2 * m] >> (8 * a)) & 255u;
          const uint32_t hi = (uint32_t)(v[2 * m + 1] >> (8 * a)) & 255u;
          const uint32_t hv = 0x64006400u | lo | (hi << 16);
          uint32_t r;
          asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(hv), "r"(0x64806480u));
          h[m] = r;
        }
        __stcs(row + (uint64_t)a * dpad, make_uint4(h[0], h[1], h[2], h[3]));
      }
    }
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

// Scratch per slot of the query multiples and the slots per launch range:
// byte-interleaved multiples (8 bytes per digit row and dimension) for tiles
// 0, 1, fp16 digit rows (16 bytes) for the TMA-fed tiles 2..8; the range is
// capped by tune[5] MiB, a multiple of 2 (slot pairs) or 4 (slot quads,
// tiles 6..8), at least that and at most N.
void batched_slot_range(const PrimeSet& P, uint32_t B, uint32_t d, const uint32_t tune[7],
                        uint64_t* per_slot, uint64_t* slots) {
  const uint32_t dpad = (d + 7) / 8 * 8;
  const bool tma_b = tune[6] >= 2, quads = tune[6] >= 6;
  const uint64_t ps = (uint64_t)P.L * 2 * B * dpad * 8 * (tma_b ? 16 : 8);
  uint64_t S = ((uint64_t)tune[5] << 20) / ps;
  S &= quads ? ~3ull : ~1ull;
  if (S < (quads ? 4u : 2u)) S = quads ? 4 : 2;
  if (S > P.N) S = P.N;
  *per_slot = ps;
  *slots = S;
}

size_t batched_scratch_bytes(const PrimeSet& P, uint32_t B, uint32_t d, const uint32_t tune[7]) {
  uint64_t ps = 0, S = 0;
  batched_slot_range(P, B, d, tune, &ps, &S);
  return (size_t)(ps * S);
}

size_t batched_limb_bytes(uint32_t L, uint32_t N, uint64_t K, uint32_t d) {
  const uint32_t dpad = (d + 7) / 8 * 8;
  return (size_t)L * N * K * 8ull * dpad * 2;
}

cudaError_t launch_wait_selftest(int* err, uint32_t limit_ms, int device, cudaStream_t st) {
  int khz = 0;
  cudaError_t e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
  if (e != cudaSuccess) return e;
  const unsigned long long cycles = (unsigned long long)limit_ms * (unsigned long long)(khz > 0 ? khz : 2000000);
  wait_selftest_kernel<<<1, 32, 0, st>>>(err, cycles);
  return cudaGetLastError();
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
                               const uint32_t tune[7], cudaStream_t st) {
  BatchArgs A;
  memset(&A, 0, sizeof(A));
  A.sleep_tma = tune[0];
  A.sleep_mma = tune[1];
  A.sleep_prod = tune[2];
  A.sleep_epi = tune[3];
  A.prefetch_units = tune[4];
  A.plimb = plimb;
  A.out = out;
  // 2: 32-byte aligned, 1: 16-byte aligned (paired / quad stores)
  A.out16 = (reinterpret_cast<uintptr_t>(out) & 31) == 0 ? 2u : (reinterpret_cast<uintptr_t>(out) & 15) == 0 ? 1u : 0u;
  A.err = err;
  A.B = B;
  A.d = d;
  A.dpad = (d + 7) / 8 * 8;
  A.K = (uint32_t)K;
  // tile shape: 0..3: bit 0 = SM pair (256 blocks) instead of one SM (128
  // blocks); bit 1 = query digits by TMA from fp16 rows instead of producer
  // warps.  4, 5: one SM per tile, TMA-fed, in clusters of 2 or 4 CTAs that
  // share each query tile by multicast.
  // 6, 7: one SM per tile, TMA-fed, four slots per CTA with 32-byte output
  // stores (batched_mac_quad_kernel), alone or in clusters of 2.
  // 8: the four-slot epilogue on SM pairs (batched_mac_pairq_kernel).
  const uint32_t tile = tune[6];
  const bool use_pair = tile < 4 && (tile & 1) != 0;
  const bool pairq = tile == 8;
  const bool tma_b = tile >= 2;
  const bool quads = tile >= 6;
  A.QT = (2 * B + kQG - 1) / kQG;
  A.KT = (uint32_t)(use_pair || pairq ? (K + 2 * pair::kBM - 1) / (2 * pair::kBM) : (K + kBM - 1) / kBM);
  // tile 7 on an odd number of database tiles runs as tile 6 rather than
  // padding a whole tile of zeros per cluster
  const int CL = tile == 4 ? 2 : tile == 5 ? 4 : (tile == 7 && A.KT % 2 == 0) ? 2 : 1;
  A.KT = (A.KT + CL - 1) / CL * CL;  // whole clusters (tiles past K load zeros and store nothing)
  A.chunks = A.dpad / 8;
  W256 W;
  memset(&W, 0, sizeof(W));
  for (uint32_t j = 0; j < P.L; ++j) {
    uint64_t w = 1 % P.q[j];
    for (int a = 0; a < 8; ++a) {
      A.w256[j][a] = w;
      A.w256_shoup[j][a] = shoup_of(w, P.q[j]);
      W.w[j][a] = w;
      W.ws[j][a] = A.w256_shoup[j][a];
      w = (uint64_t)(((u128)w * 256) % P.q[j]);
    }
    A.r256_shoup[j] = shoup_of(256 % P.q[j], P.q[j]);
    A.w32[j] = (uint64_t)(((u128)1 << 32) % P.q[j]);
    A.w32_shoup[j] = shoup_of(A.w32[j], P.q[j]);
    A.mu64[j] = (uint64_t)(((u128)1 << 64) / P.q[j]);
    A.lo_bias[j] = ((1ull << 49) + P.q[j] - 1) / P.q[j] * P.q[j];
  }
  // slot ranges bound the scratch of the query multiples (tune[5] MiB, at
  // least one slot's worth)
  uint64_t per_slot = 0, S = 0;
  batched_slot_range(P, B, d, tune, &per_slot, &S);
  const size_t smem = use_pair ? (size_t)pair::kSmem : pairq ? (size_t)pq::kSmem
                    : quads ? (size_t)quad::kSmem : (size_t)kSmem1;
  // kernel attributes and the number of co-resident CTA pairs (clusters of 2
  // need two SMs of one GPC) are set up once per device, outside any capture
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex setup_mu;
  static int pairs_resident_dev[64] = {};
  static int pairq_resident_dev[64] = {};
  static int clusters_resident_dev[64][3] = {};   // clusters of 2 and of 4 (tiles 4, 5), quad clusters of 2 (7)
  static bool configured_dev[64] = {};
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int pairs_resident = 0, clusters_resident = 0;
  {
    std::lock_guard<std::mutex> lock(setup_mu);
    if (!configured_dev[dev]) {
      // residency on the whole device (the cap below applies per launch)
      int dev_sms = 0;
      e = cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      const void* cluster_kernels[2] = {(const void*)batched_mac_kernel<true, 2>,
                                        (const void*)batched_mac_kernel<true, 4>};
      for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
        e = cudaFuncSetAttribute(cluster_kernels[c], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem1);
        if (e != cudaSuccess) break;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2u << c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(dev_sms / (2 << c) * (2 << c)));
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = kSmem1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(&clusters_resident_dev[dev][c], cluster_kernels[c], &cfg);
      }
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(batched_mac_pair_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)pair::kSmem);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batched_mac_pair_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair::kSmem);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batched_mac_kernel<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmem1);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batched_mac_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmem1);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batched_mac_quad_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)quad::kSmem);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batched_mac_quad_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)quad::kSmem);
      if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(dev_sms / 2 * 2));
        cfg.blockDim = dim3(quad::kThreads);
        cfg.dynamicSmemBytes = quad::kSmem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(&clusters_resident_dev[dev][2], batched_mac_quad_kernel<2>, &cfg);
      }
      if (e != cudaSuccess) return e;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(2 * (unsigned)(dev_sms / 2));
      cfg.blockDim = dim3(pair::kThreads);
      cfg.dynamicSmemBytes = pair::kSmem;
      e = cudaOccupancyMaxActiveClusters(&pairs_resident_dev[dev], batched_mac_pair_kernel<false>, &cfg);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(batched_mac_pairq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)pq::kSmem);
      if (e != cudaSuccess) return e;
      cfg.blockDim = dim3(pq::kThreads);
      cfg.dynamicSmemBytes = pq::kSmem;
      e = cudaOccupancyMaxActiveClusters(&pairq_resident_dev[dev], batched_mac_pairq_kernel, &cfg);
      if (e != cudaSuccess) return e;
      configured_dev[dev] = true;
    }
    pairs_resident = pairq ? pairq_resident_dev[dev] : pairs_resident_dev[dev];
    if (CL > 1) clusters_resident = clusters_resident_dev[dev][quads ? 2 : CL == 2 ? 0 : 1];
  }
  if ((use_pair || pairq) && pairs_resident < 1) return cudaErrorInvalidConfiguration;
  if (CL > 1 && clusters_resident < 1) return cudaErrorInvalidConfiguration;
  // an SM cap (sms > 0) bounds the persistent grid; at least one CTA pair or
  // cluster still runs
  if (sms > 0) {
    const int cap2 = sms / 2 > 0 ? sms / 2 : 1, capc = sms / CL > 0 ? sms / CL : 1;
    if (pairs_resident > cap2) pairs_resident = cap2;
    if (CL > 1 && clusters_resident > capc) clusters_resident = capc;
  }
  PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  e = get_encode(&enc);
  if (e != cudaSuccess) return e;
  uint64_t* scratch = nullptr;
  e = cudaMallocAsync(&scratch, per_slot * S, st);
  if (e != cudaSuccess) return e;
  CUtensorMap m;
  memcpy(&m, map, sizeof(m));
  for (uint64_t s0 = 0; s0 < P.N && e == cudaSuccess; s0 += S) {
    const uint32_t cnt = (uint32_t)(s0 + S <= P.N ? S : P.N - s0);
    A.s_begin = (uint32_t)s0;
    A.s_count = cnt;
    A.xm = scratch;
    A.xh = reinterpret_cast<const uint16_t*>(scratch);
    // one-SM tiles count slot pairs or quads (all in one CTA; per cluster of
    // CL database tiles), SM pairs single slots
    A.units = (uint64_t)P.L * (use_pair ? cnt : quads ? cnt / 4 : cnt / 2) * (A.KT / CL) * A.QT;
    if (A.units >= (1ull << 31)) { e = cudaErrorInvalidValue; break; }
    const dim3 xgrid((cnt + 31) / 32, A.dpad / 8, P.L * 2 * B);
    CUtensorMap xmap;
    CUresult cr = CUDA_SUCCESS;
    if (tma_b) {
      expand_query_f16_kernel<<<dim3((cnt + 3) / 4, P.L), 256, 0, st>>>(P, ct, B, d, A.dpad, (uint32_t)s0, cnt,
                                                                      W, reinterpret_cast<uint4*>(scratch));
      // fp16 digit rows as a tensor [L S'][16 B][8 dpad]; boxes of 64
      // contraction columns x 256 rows (one SM) or 128 rows (each CTA of a pair)
      const cuuint64_t dims[3] = {8ull * A.dpad, 16ull * B, (cuuint64_t)P.L * cnt};
      const cuuint64_t strides[2] = {16ull * A.dpad, 16ull * B * 16ull * A.dpad};
      const cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)(use_pair || pairq ? pair::kBNh : kBN / CL), 1};
      const cuuint32_t estr[3] = {1, 1, 1};
      cr = enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, scratch, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
      expand_query_kernel<<<xgrid, 256, 0, st>>>(P, ct, B, d, A.dpad, (uint32_t)s0, cnt, W,
                                                 reinterpret_cast<ulonglong2*>(scratch));
      if (use_pair) {
        // query multiples of this range as a tensor: [L S'][2B][dpad / 8][64 u64],
        // boxes of 16 row groups x one 8-dimension block (8 KB)
        const cuuint64_t dims[4] = {64, A.dpad / 8, 2ull * B, (cuuint64_t)P.L * cnt};
        const cuuint64_t strides[3] = {512, 64ull * A.dpad, 128ull * B * A.dpad};
        const cuuint32_t box[4] = {64, 1, (cuuint32_t)pair::kQGh, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        cr = enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, scratch, dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      } else {
        memcpy(&xmap, &m, sizeof(m));   // unused by the producer-fed tile
      }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    if (cr != CUDA_SUCCESS) { e = cudaErrorInvalidValue; break; }
    if (use_pair) {
      uint64_t clusters = (uint64_t)pairs_resident;
      if (clusters > A.units) clusters = A.units;
      if (tma_b)
        batched_mac_pair_kernel<true><<<(unsigned)(2 * clusters), pair::kThreads, smem, st>>>(m, xmap, P, A);
      else
        batched_mac_pair_kernel<false><<<(unsigned)(2 * clusters), pair::kThreads, smem, st>>>(m, xmap, P, A);
    } else if (pairq) {
      uint64_t clusters = (uint64_t)pairs_resident;
      if (clusters > A.units) clusters = A.units;
      batched_mac_pairq_kernel<<<(unsigned)(2 * clusters), pq::kThreads, smem, st>>>(m, xmap, P, A);
    } else if (quads) {
      uint64_t clusters = CL > 1 ? (uint64_t)clusters_resident : (uint64_t)(sms > 0 ? sms : 148);
      if (clusters > A.units) clusters = A.units;
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)CL;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)(clusters * CL));
      cfg.blockDim = dim3(quad::kThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = st;
      cfg.attrs = at;
      cfg.numAttrs = CL > 1 ? 1 : 0;
      if (CL == 2) e = cudaLaunchKernelEx(&cfg, batched_mac_quad_kernel<2>, m, xmap, P, A);
      else e = cudaLaunchKernelEx(&cfg, batched_mac_quad_kernel<1>, m, xmap, P, A);
      if (e != cudaSuccess) break;
    } else if (CL > 1) {
      uint64_t clusters = (uint64_t)clusters_resident;
      if (clusters > A.units) clusters = A.units;
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)CL;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)(clusters * CL));
      cfg.blockDim = dim3(kThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = st;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if (CL == 2) e = cudaLaunchKernelEx(&cfg, batched_mac_kernel<true, 2>, m, xmap, P, A);
      else e = cudaLaunchKernelEx(&cfg, batched_mac_kernel<true, 4>, m, xmap, P, A);
      if (e != cudaSuccess) break;
    } else {
      uint64_t grid = (uint64_t)(sms > 0 ? sms : 148);
      if (grid > A.units) grid = A.units;
      if (tma_b)
        batched_mac_kernel<true, 1><<<(unsigned)grid, kThreads, smem, st>>>(m, xmap, P, A);
      else
        batched_mac_kernel<false, 1><<<(unsigned)grid, kThreads, smem, st>>>(m, xmap, P, A);
    }
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(scratch, st);
  return e != cudaSuccess ? e : e2;
}

}  // namespace sanns
