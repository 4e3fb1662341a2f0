// K2: the ct x pt multiply-accumulate of the distance step (Pi_ls step 3,
// f_k = sum_i CMult(c_i, p_ik)).  In the NTT domain CMult is slot-wise, so per
// (query b, block k, component c, prime j, slot s)
//     acc = sum_i ct[b][i][c][j][s] * pt[k][j][i][s]  mod q_j.
//
// The encoded database (d L 8 bytes per point) is streamed from HBM exactly
// once per query; the query ciphertext tile for 32 SPL slots stays in shared
// memory while every block k of that tile streams past it (each warp takes a
// different k).
//
// Arithmetic: the query values are put in Montgomery form (x 2^64 mod q) and
// both operands are split into 30-bit halves x = x1 2^30 + x0 (the database
// is stored with its halves in separate 32-bit words, so only the query tile
// is split, once per tile).  The four
// partial products go into four 64-bit accumulators with one 32x32->64
// multiply-add each; 16 products of (2^30 - 1)^2 fit in 64 bits, so every 16
// dimensions the partials are folded into an exact 128-bit sum R.  R < d q^2
// < 2^128 for d <= 224, q < 2^60, and one Montgomery reduction of R gives
// sum_i ct pt mod q below 15 q, finished by four conditional subtractions.
//
// Launch variants (slots per lane, dimensions per load batch, threads, CTAs
// per SM) trade registers for loads in flight; sanns_autotune_mac times them.
// Pair variants (QN = 2) hold two queries' ct tiles and use every database
// word they load for both, halving the database traffic of a multi-query
// call; calls with B >= 2 run the pair sibling of the selected variant.
#include "internal.h"

namespace sanns {

namespace {

constexpr uint32_t kMask30 = (1u << 30) - 1;

struct MacArgs {
  const uint64_t* ct;  // [B][d][2][L][N], NTT form
  const uint64_t* pt;  // [K][L][d][N], NTT form, split30 format (30-bit halves in the two words)
  uint64_t* out;       // [B][K][2][L][N]
  uint64_t K;
  uint64_t total;      // ceil(B / QN) L (N / tile) K work items (tile, block)
  uint32_t d;
  uint32_t B;
};

// acc += a b for a 64-bit sum that cannot overflow: the low product word
// added with a carry out, the high word with that carry in.
__device__ __forceinline__ void mad_acc(uint64_t& acc, uint32_t a, uint32_t b) {
  asm("{\n\t.reg .u32 lo, hi;\n\t"
      "mov.b64 {lo, hi}, %0;\n\t"
      "mad.lo.cc.u32 lo, %1, %2, lo;\n\t"
      "madc.hi.u32 hi, %1, %2, hi;\n\t"
      "mov.b64 %0, {lo, hi};\n\t}"
      : "+l"(acc)
      : "r"(a), "r"(b));
}

__device__ __forceinline__ void mac4(uint64_t& aL, uint64_t& aM1, uint64_t& aM2, uint64_t& aH,
                                     uint32_t xl, uint32_t xh, uint32_t yl, uint32_t yh) {
  mad_acc(aL, xl, yl);
  mad_acc(aM1, xh, yl);
  mad_acc(aM2, xl, yh);
  mad_acc(aH, xh, yh);
}

template <int SPL>
struct PtVec;
template <>
struct PtVec<1> {
  typedef unsigned long long T;
  static __device__ __forceinline__ T load(const uint64_t* p) {
    return __ldcs(reinterpret_cast<const unsigned long long*>(p));
  }
  static __device__ __forceinline__ T zero() { return 0ull; }
  static __device__ __forceinline__ uint64_t get(const T& v, int) { return v; }
};
template <>
struct PtVec<2> {
  typedef ulonglong2 T;
  static __device__ __forceinline__ T load(const uint64_t* p) {
    return __ldcs(reinterpret_cast<const ulonglong2*>(p));
  }
  static __device__ __forceinline__ T zero() { return make_ulonglong2(0, 0); }
  static __device__ __forceinline__ uint64_t get(const T& v, int s) { return s ? v.y : v.x; }
};

// ct tile in shared memory, per (dimension i, lane): for SPL = 1 one uint4
// {c0 lo, c0 hi, c1 lo, c1 hi} per query of the pass (QN of them); for
// SPL = 2 two uint4 (c0, c1), each {lo(s0), hi(s0), lo(s1), hi(s1)}.
template <int SPL, int UNR, int THREADS, int MINB, int QN = 1>
__global__ void __launch_bounds__(THREADS, MINB) mac_kernel(PrimeSet P, MacArgs A) {
  static_assert(QN == 1 || SPL == 1, "query pairs use one slot per lane");
  extern __shared__ uint4 cts[];
  constexpr int WARPS = THREADS / 32;
  constexpr uint32_t TILE = 32 * SPL;
  constexpr int NOUT = 2 * SPL * QN;  // (query, c, slot) outputs per lane
  typedef PtVec<SPL> V;
  const uint32_t N = P.N, L = P.L, d = A.d;
  const uint32_t tiles = N / TILE;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // Work is split into rounds: a run of K blocks (one tile) is ceil(K / WARPS)
  // rounds of at most WARPS blocks, one per warp.  Each CTA takes an even
  // share of the rounds, so its item range starts and ends on round
  // boundaries and no run is cut into pieces that each pay a partial round.
  const uint64_t rounds_per_run = (A.K + WARPS - 1) / WARPS;
  const uint64_t rounds = A.total / A.K * rounds_per_run;
  auto item_of_round = [&](uint64_t r) -> uint64_t {
    const uint64_t in_run = (r % rounds_per_run) * WARPS;
    return r / rounds_per_run * A.K + (in_run < A.K ? in_run : A.K);
  };
  const uint64_t w_begin = item_of_round(blockIdx.x * rounds / gridDim.x);
  const uint64_t w_end = item_of_round((blockIdx.x + 1) * rounds / gridDim.x);

  uint64_t w = w_begin;
  while (w < w_end) {
    const uint64_t u = w / A.K;                     // (b L + j) tiles + st
    const uint64_t k_first = w - u * A.K;
    const uint64_t run_end = min(w_end, (u + 1) * A.K);
    const uint32_t nk = (uint32_t)(run_end - w);
    const uint32_t st = (uint32_t)(u % tiles);
    const uint32_t j = (uint32_t)((u / tiles) % L);
    const uint64_t b = u / ((uint64_t)tiles * L) * QN;  // first query of the pass
    const bool pair = QN == 2 && b + 1 < A.B;            // a second query exists
    const uint64_t q = P.q[j];

    __syncthreads();  // previous tile fully consumed
    for (uint32_t e = threadIdx.x; e < d * 2 * 32 * QN; e += THREADS) {
      const uint32_t l = e & 31, ci = e >> 5, c = ci & 1, qi = (ci >> 1) % QN, i = (ci >> 1) / QN;
      const uint64_t bq = b + (pair ? qi : 0);
      const uint64_t* src = A.ct + ((((bq * d + i) * 2 + c) * L + j) * N) + st * TILE + SPL * l;
      uint64_t m[SPL];
#pragma unroll
      for (int s = 0; s < SPL; ++s) m[s] = mul_shoup(src[s], P.r64[j], P.r64_shoup[j], q);
      if (SPL == 1) {
        uint32_t* dst = reinterpret_cast<uint32_t*>(&cts[(i * QN + qi) * 32 + l]) + 2 * c;
        dst[0] = (uint32_t)m[0] & kMask30;
        dst[1] = (uint32_t)(m[0] >> 30);
      } else {
        cts[(i * 2 + c) * 32 + l] = make_uint4((uint32_t)m[0] & kMask30, (uint32_t)(m[0] >> 30),
                                               (uint32_t)m[SPL - 1] & kMask30,
                                               (uint32_t)(m[SPL - 1] >> 30));
      }
    }
    __syncthreads();

    for (uint32_t kk = warp; kk < nk; kk += WARPS) {
      const uint64_t k = k_first + kk;
      const uint64_t* p = A.pt + ((k * L + j) * d) * N + st * TILE + SPL * lane;
      u128 R[NOUT];
      uint64_t aL[NOUT], aM1[NOUT], aM2[NOUT], aH[NOUT];
#pragma unroll
      for (int o = 0; o < NOUT; ++o) { R[o] = 0; aL[o] = aM1[o] = aM2[o] = aH[o] = 0; }

      for (uint32_t i0 = 0; i0 < d; i0 += 16) {
#pragma unroll
        for (int h = 0; h < 16 / UNR; ++h) {
          typename V::T pv[UNR];
#pragma unroll
          for (int v = 0; v < UNR; ++v) {
            const uint32_t i = i0 + UNR * h + v;
            pv[v] = i < d ? V::load(p + (uint64_t)i * N) : V::zero();
          }
#pragma unroll
          for (int v = 0; v < UNR; ++v) {
            const uint32_t i = i0 + UNR * h + v;
            const uint32_t ii = i < d ? i : d - 1;  // beyond d the pt values are zero
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
              const uint64_t y = V::get(pv[v], s);
              const uint32_t yl = (uint32_t)y, yh = (uint32_t)(y >> 32);  // stored split
              if (SPL == 1) {
#pragma unroll
                for (int qi = 0; qi < QN; ++qi) {
                  const uint4 x = cts[(ii * QN + qi) * 32 + lane];
                  mac4(aL[2 * qi], aM1[2 * qi], aM2[2 * qi], aH[2 * qi], x.x, x.y, yl, yh);  // c0
                  mac4(aL[2 * qi + 1], aM1[2 * qi + 1], aM2[2 * qi + 1], aH[2 * qi + 1], x.z, x.w, yl,
                       yh);  // c1
                }
              } else {
                const uint4 x0 = cts[(ii * 2 + 0) * 32 + lane];
                const uint4 x1 = cts[(ii * 2 + 1) * 32 + lane];
                const uint32_t c0l = s ? x0.z : x0.x, c0h = s ? x0.w : x0.y;
                const uint32_t c1l = s ? x1.z : x1.x, c1h = s ? x1.w : x1.y;
                mac4(aL[s], aM1[s], aM2[s], aH[s], c0l, c0h, yl, yh);                  // c0
                mac4(aL[2 + s], aM1[2 + s], aM2[2 + s], aH[2 + s], c1l, c1h, yl, yh);  // c1
              }
            }
          }
        }
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
          const u128 m = (u128)aM1[o] + aM2[o];
          R[o] += (u128)aL[o] + (m << 30) + ((u128)aH[o] << 60);
          aL[o] = aM1[o] = aM2[o] = aH[o] = 0;
        }
      }
      const uint64_t qn = P.q_neg_inv[j];
      uint64_t r[NOUT];
#pragma unroll
      for (int o = 0; o < NOUT; ++o) r[o] = reduce_below_16q(redc128(R[o], q, qn), q);
      uint64_t* o0 = A.out + (((b * A.K + k) * 2 + 0) * L + j) * N + st * TILE + SPL * lane;
      uint64_t* o1 = A.out + (((b * A.K + k) * 2 + 1) * L + j) * N + st * TILE + SPL * lane;
      if (SPL == 1) {
        // query qi's c0 at r[2 qi], c1 at r[2 qi + 1]
        *o0 = r[0];
        *o1 = r[1];
        if (QN == 2 && pair) {
          const uint64_t step = A.K * 2 * L * N;  // the next query's outputs
          o0[step] = r[2 % NOUT];
          o1[step] = r[3 % NOUT];
        }
      } else {
        *reinterpret_cast<ulonglong2*>(o0) = make_ulonglong2(r[0], r[1]);
        *reinterpret_cast<ulonglong2*>(o1) = make_ulonglong2(r[2 % NOUT], r[3 % NOUT]);
      }
    }
    w = run_end;
  }
}

// Few work items (one query over a small database): one CTA per (tile,
// block) item, its eight warps splitting the d dimensions, so that each warp's
// chain of dependent loads is d/8 long instead of d.  Each lane reads its two
// slots' ct values straight from global memory (Montgomery form and 30-bit
// halves formed in registers) beside the database words; the warps' exact
// 128-bit partial sums meet in shared memory and warp 0 reduces them.
template <int SPL, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) mac_split_kernel(PrimeSet P, MacArgs A) {
  static_assert(SPL == 2, "two slots per lane");
  constexpr int WARPS = THREADS / 32;
  constexpr uint32_t TILE = 32 * SPL;
  constexpr int NOUT = 2 * SPL;
  constexpr int BATCH = 8;                 // dimensions whose loads are in flight together
  __shared__ ulonglong2 red[WARPS][NOUT][32];
  const uint32_t N = P.N, L = P.L, d = A.d;
  const uint32_t tiles = N / TILE;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t w = blockIdx.x; w < A.total; w += gridDim.x) {
    const uint64_t u = w / A.K, k = w - u * A.K;
    const uint32_t st = (uint32_t)(u % tiles);
    const uint32_t j = (uint32_t)((u / tiles) % L);
    const uint64_t b = u / ((uint64_t)tiles * L);
    const uint64_t q = P.q[j], r64 = P.r64[j], r64s = P.r64_shoup[j];
    const uint32_t per = (d + WARPS - 1) / WARPS;
    const uint32_t i_begin = warp * per, i_end = min(d, i_begin + per);
    const uint64_t* p = A.pt + ((k * L + j) * d) * N + st * TILE + SPL * lane;
    const uint64_t* c = A.ct + (b * d * 2 * L + j) * N + st * TILE + SPL * lane;  // dimension 0, c0
    u128 R[NOUT];
    uint64_t aL[NOUT], aM1[NOUT], aM2[NOUT], aH[NOUT];
#pragma unroll
    for (int o = 0; o < NOUT; ++o) { R[o] = 0; aL[o] = aM1[o] = aM2[o] = aH[o] = 0; }
    uint32_t since_fold = 0;
    for (uint32_t i0 = i_begin; i0 < i_end; i0 += BATCH) {
      ulonglong2 pv[BATCH], c0v[BATCH], c1v[BATCH];
#pragma unroll
      for (int v = 0; v < BATCH; ++v) {
        const uint32_t i = i0 + v;
        const bool in = i < i_end;
        pv[v] = in ? __ldcs(reinterpret_cast<const ulonglong2*>(p + (uint64_t)i * N)) : make_ulonglong2(0, 0);
        c0v[v] = in ? __ldg(reinterpret_cast<const ulonglong2*>(c + (uint64_t)i * 2 * L * N))
                    : make_ulonglong2(0, 0);
        c1v[v] = in ? __ldg(reinterpret_cast<const ulonglong2*>(c + ((uint64_t)i * 2 + 1) * L * N))
                    : make_ulonglong2(0, 0);
      }
#pragma unroll
      for (int v = 0; v < BATCH; ++v) {
        if (i0 + v >= i_end) break;
        if (since_fold == 16) {  // 16 products of (2^30 - 1)^2 fill a 64-bit sum
#pragma unroll
          for (int o = 0; o < NOUT; ++o) {
            const u128 m = (u128)aM1[o] + aM2[o];
            R[o] += (u128)aL[o] + (m << 30) + ((u128)aH[o] << 60);
            aL[o] = aM1[o] = aM2[o] = aH[o] = 0;
          }
          since_fold = 0;
        }
        const uint64_t y[SPL] = {pv[v].x, pv[v].y};
        const uint64_t x0[SPL] = {mul_shoup(c0v[v].x, r64, r64s, q), mul_shoup(c0v[v].y, r64, r64s, q)};
        const uint64_t x1[SPL] = {mul_shoup(c1v[v].x, r64, r64s, q), mul_shoup(c1v[v].y, r64, r64s, q)};
#pragma unroll
        for (int s = 0; s < SPL; ++s) {
          const uint32_t yl = (uint32_t)y[s], yh = (uint32_t)(y[s] >> 32);  // stored split
          mac4(aL[s], aM1[s], aM2[s], aH[s], (uint32_t)x0[s] & kMask30, (uint32_t)(x0[s] >> 30), yl, yh);
          mac4(aL[2 + s], aM1[2 + s], aM2[2 + s], aH[2 + s], (uint32_t)x1[s] & kMask30,
               (uint32_t)(x1[s] >> 30), yl, yh);
        }
        ++since_fold;
      }
    }
#pragma unroll
    for (int o = 0; o < NOUT; ++o) {
      const u128 m = (u128)aM1[o] + aM2[o];
      R[o] += (u128)aL[o] + (m << 30) + ((u128)aH[o] << 60);
      red[warp][o][lane] = make_ulonglong2((uint64_t)R[o], (uint64_t)(R[o] >> 64));
    }
    __syncthreads();
    if (warp == 0) {
      const uint64_t qn = P.q_neg_inv[j];
      uint64_t r[NOUT];
#pragma unroll
      for (int o = 0; o < NOUT; ++o) {
        u128 S = 0;
#pragma unroll
        for (int wi = 0; wi < WARPS; ++wi) {
          const ulonglong2 h = red[wi][o][lane];
          S += ((u128)h.y << 64) | h.x;
        }
        r[o] = reduce_below_16q(redc128(S, q, qn), q);
      }
      uint64_t* o0 = A.out + (((b * A.K + k) * 2 + 0) * L + j) * N + st * TILE + SPL * lane;
      uint64_t* o1 = A.out + (((b * A.K + k) * 2 + 1) * L + j) * N + st * TILE + SPL * lane;
      *reinterpret_cast<ulonglong2*>(o0) = make_ulonglong2(r[0], r[1]);
      *reinterpret_cast<ulonglong2*>(o1) = make_ulonglong2(r[2], r[3]);
    }
    __syncthreads();  // red[] is reused by the next item
  }
}

struct MacVariant {
  void (*fn)(PrimeSet, MacArgs);
  int spl, threads, ctas_per_sm, qn;
  int pair_sibling;  // the variant run for calls with B >= 2 (-1: itself)
  const char* name;
  bool split = false;  // mac_split_kernel: one CTA per item, no shared ct tile
};

const MacVariant kVariants[] = {
    {mac_kernel<2, 8, 512, 1>, 2, 512, 1, 1, 4, "spl2_unr8_512x1"},
    {mac_kernel<1, 16, 256, 3>, 1, 256, 3, 1, 5, "spl1_unr16_256x3"},
    {mac_kernel<1, 8, 256, 3>, 1, 256, 3, 1, 5, "spl1_unr8_256x3"},
    {mac_kernel<1, 16, 384, 2>, 1, 384, 2, 1, 4, "spl1_unr16_384x2"},
    {mac_kernel<1, 8, 512, 1, 2>, 1, 512, 1, 2, -1, "pair_unr8_512x1"},
    {mac_kernel<1, 8, 256, 2, 2>, 1, 256, 2, 2, -1, "pair_unr8_256x2"},
    {mac_split_kernel<2, 256>, 2, 256, 1, 1, -1, "split_d_256x1", true},
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

}  // namespace

int mac_num_variants() { return kNumVariants; }
const char* mac_variant_name(int v) { return (v >= 0 && v < kNumVariants) ? kVariants[v].name : ""; }

cudaError_t launch_mac(const PrimeSet& P, const uint64_t* ct, const uint64_t* pt, uint32_t B,
                       uint32_t d, uint64_t K, uint64_t* out, int sms, int variant,
                       cudaStream_t st) {
  if (variant < 0 || variant >= kNumVariants) return cudaErrorInvalidValue;
  if (B >= 2 && kVariants[variant].pair_sibling >= 0) variant = kVariants[variant].pair_sibling;
  const MacVariant& V = kVariants[variant];
  const uint32_t tile = 32u * V.spl;
  MacArgs A;
  A.ct = ct;
  A.pt = pt;
  A.out = out;
  A.K = K;
  A.d = d;
  A.B = B;
  A.total = (uint64_t)((B + V.qn - 1) / V.qn) * P.L * (P.N / tile) * K;
  if (A.total == 0) return cudaSuccess;
  if (V.split) {
    // one CTA per item up to eight per SM (the grid loops beyond that)
    uint64_t grid = (uint64_t)(sms > 0 ? sms : 148) * 8;
    if (grid > A.total) grid = A.total;
    V.fn<<<(unsigned)grid, V.threads, 0, st>>>(P, A);
    return cudaGetLastError();
  }
  const size_t smem = sizeof(uint4) * 32 * d * V.spl * V.qn;
  // shared-memory opt-in, once per (variant, device)
  cudaError_t e = ensure_smem_attr((const void*)V.fn, smem > 48 * 1024 ? smem : 48 * 1024);
  if (e != cudaSuccess) return e;
  int per_sm = V.ctas_per_sm;
  // fewer co-resident CTAs when the ct tile is large
  while (per_sm > 1 && smem * per_sm > 220 * 1024) --per_sm;
  uint64_t grid = (uint64_t)(sms > 0 ? sms : 148) * per_sm;
  if (grid > A.total) grid = A.total;
  V.fn<<<(unsigned)grid, V.threads, smem, st>>>(P, A);
  return cudaGetLastError();
}

}  // namespace sanns
