// Device-side building blocks of the SANNS encrypted-distance library:
// 64-bit modular arithmetic (Shoup and Montgomery forms), ChaCha20 draws and
// the context structures every kernel receives by value.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sanns.h"

namespace sanns {

typedef unsigned __int128 u128;

constexpr int kMaxPrimes = 4;
constexpr uint32_t kMaxN = 16384;
constexpr uint32_t kMinN = 64;
constexpr uint32_t kMaxD = 224;   // ct tile of the MAC kernel lives in shared memory

// Stream purposes of the counter-based generator (ChaCha20, RFC 8439).
enum : uint32_t {
  kPurposeSk = 1, kPurposeA = 2, kPurposeE = 3, kPurposeMask = 4,
  // circuit privacy: public key (client), re-randomisation and flooding (server)
  kPurposeAPk = 5, kPurposeEPk = 6, kPurposeU = 7, kPurposeE2 = 8, kPurposeFloodLo = 9,
  kPurposeFloodHi = 10
};

// Constants of the flooding term (circuit privacy), per prime.
struct PrivacyConsts {
  uint64_t q_barrett[kMaxPrimes];   // floor(2^64 / q_j)
  uint64_t two_f[kMaxPrimes];       // 2^F mod q_j
};

// Modulus switching of responses from q_0 .. q_{L-1} down to q_0 (modswitch.cu):
// Garner constants of the dropped primes q_1 .. q_{L-1}, by value.
struct ModSwitchConsts {
  uint64_t g[kMaxPrimes][kMaxPrimes];   // g[i][m] = q_1 .. q_{m-1} mod q_i (m < i)
  uint64_t gs[kMaxPrimes][kMaxPrimes];
  uint64_t ginv[kMaxPrimes];            // (q_1 .. q_{i-1})^-1 mod q_i
  uint64_t ginvs[kMaxPrimes];
  uint64_t h[kMaxPrimes];               // mixed-radix digits of (P - 1) / 2, P = q_1 .. q_{L-1}
  uint64_t w0[kMaxPrimes];              // q_1 .. q_{m-1} mod q_0
  uint64_t w0s[kMaxPrimes];
  uint64_t p0;                          // P mod q_0
  uint64_t pinv0, pinv0s;               // P^-1 mod q_0
};

// Per-prime constants, passed to kernels by value.
struct PrimeSet {
  uint32_t N, logN, L;
  uint32_t norms_below_t;           // every stored ||p||^2 is below t (d 255^2 < t)
  uint64_t t;                       // plaintext modulus
  uint64_t t_barrett;               // floor(2^64 / t)
  uint64_t two64_mod_t;             // 2^64 mod t
  uint64_t q[kMaxPrimes];
  uint64_t q_neg_inv[kMaxPrimes];   // -q^-1 mod 2^64 (Montgomery REDC)
  uint64_t r64[kMaxPrimes];         // 2^64 mod q
  uint64_t r64_shoup[kMaxPrimes];
  uint64_t delta[kMaxPrimes];       // floor(Q / t) mod q
  uint64_t delta_shoup[kMaxPrimes];
  uint64_t n_inv[kMaxPrimes];       // N^-1 mod q
  uint64_t n_inv_shoup[kMaxPrimes];
  uint64_t crt_inv[kMaxPrimes];     // (Q / q_j)^-1 mod q_j
  uint64_t crt_inv_shoup[kMaxPrimes];
  uint64_t last_inv[kMaxPrimes];    // psi^-brv(1) N^-1 mod q: last inverse stage with N^-1
  uint64_t last_inv_shoup[kMaxPrimes];
  uint64_t delta_w1[kMaxPrimes];    // Delta psi^brv(1) mod q: first forward stage of Delta v
  uint64_t delta_w1_shoup[kMaxPrimes];
  // twiddles, [L][N] pairs {w, Shoup companion}: psi^brv(m) and psi^-brv(m)
  const ulonglong2* tw;
  const ulonglong2* itw;
  // Montgomery images of coordinate bytes, [L][2][256]: a 2^64 mod q and
  // b psi^brv(1) 2^64 mod q (the first forward stage of a byte polynomial)
  const uint64_t* mbyte;
};

// ------------------------------------------------------------------------
// modular arithmetic
// ------------------------------------------------------------------------
// w * y mod q, lazily in [0, 2q), for any y < 2^64, w < q < 2^62 and
// w_shoup = floor(w 2^64 / q) (Shoup's precomputed-quotient product).
__device__ __forceinline__ uint64_t mul_shoup_lazy(uint64_t y, uint64_t w, uint64_t w_shoup,
                                                   uint64_t q) {
  uint64_t qt = __umul64hi(w_shoup, y);
  return w * y - qt * q;
}

__device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t m) { return x >= m ? x - m : x; }

// w * y mod q lazily in [0, 4q), for any y < 2^64, w < q < 2^61: the Shoup
// quotient floor(y w_shoup / 2^64) is estimated from three of the four 32-bit
// partial products (the dropped low terms add less than 3 to the exact
// value), so the estimate is at most 2 below it and the remainder below 4q.
__device__ __forceinline__ uint64_t mul_shoup_lazy4(uint64_t y, uint64_t w, uint64_t w_shoup,
                                                    uint64_t q) {
  const uint32_t y0 = (uint32_t)y, y1 = (uint32_t)(y >> 32);
  const uint32_t s0 = (uint32_t)w_shoup, s1 = (uint32_t)(w_shoup >> 32);
  uint64_t qt = (uint64_t)y1 * s1 + __umulhi(y0, s1);
  qt += __umulhi(y1, s0);
  return w * y - qt * q;
}

__device__ __forceinline__ uint64_t mul_shoup(uint64_t y, uint64_t w, uint64_t w_shoup,
                                              uint64_t q) {
  return csub(mul_shoup_lazy(y, w, w_shoup, q), q);
}

// w * v mod q lazily in [0, 2q) for a 32-bit v (values mod t): the same
// Shoup quotient floor(v w_shoup / 2^64), exactly, from two 32-bit partial
// products, and a quotient below 2^32.
__device__ __forceinline__ uint64_t mul_shoup_u32_lazy(uint32_t v, uint64_t w, uint64_t w_shoup,
                                                       uint64_t q) {
  const uint64_t hi = (uint64_t)v * (uint32_t)(w_shoup >> 32) + __umulhi(v, (uint32_t)w_shoup);
  const uint32_t qt = (uint32_t)(hi >> 32);
  return (uint64_t)v * w - (uint64_t)qt * q;
}

__device__ __forceinline__ uint64_t mul_shoup_u32(uint32_t v, uint64_t w, uint64_t w_shoup, uint64_t q) {
  return csub(mul_shoup_u32_lazy(v, w, w_shoup, q), q);
}

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
  return csub(a + b, q);
}

__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
  return a >= b ? a - b : a + q - b;
}

// Montgomery reduction of a 128-bit value r < 2^64 * 2^64 - ..., returning
// (r + m q) / 2^64 with m = r_lo * (-q^-1) mod 2^64; the value is r 2^-64 mod q
// and lies below r / 2^64 + q.
__device__ __forceinline__ uint64_t redc128(u128 r, uint64_t q, uint64_t q_neg_inv) {
  uint64_t lo = (uint64_t)r, hi = (uint64_t)(r >> 64);
  uint64_t m = lo * q_neg_inv;
  uint64_t mh = __umul64hi(m, q);
  return hi + mh + (lo != 0 ? 1ull : 0ull);
}

// x mod q for x < 16 q.
__device__ __forceinline__ uint64_t reduce_below_16q(uint64_t x, uint64_t q) {
  x = csub(x, q << 3);
  x = csub(x, q << 2);
  x = csub(x, q << 1);
  return csub(x, q);
}

// x mod t for x < 2^64 with t_barrett = floor(2^64 / t): the estimate
// floor(x * t_barrett / 2^64) is at most one below floor(x / t).
__device__ __forceinline__ uint64_t mod_t64(uint64_t x, uint64_t t, uint64_t t_barrett) {
  uint64_t qt = __umul64hi(x, t_barrett);
  return csub(x - qt * t, t);
}

// (||p||^2 + r) mod t for a stored norm and a mask value r < t: one
// conditional subtraction when the norms are below t, else Barrett.
__device__ __forceinline__ uint64_t norm_plus_mask_mod_t(const PrimeSet& P, uint32_t norm, uint64_t r) {
  const uint64_t x = (uint64_t)norm + r;
  return P.norms_below_t ? csub(x, P.t) : mod_t64(x, P.t, P.t_barrett);
}

// (hi 2^64 + lo) mod t, t < 2^32.
__device__ __forceinline__ uint64_t mod_t128(uint64_t lo, uint64_t hi, const PrimeSet& P) {
  uint64_t h = mod_t64(hi, P.t, P.t_barrett);
  uint64_t l = mod_t64(lo, P.t, P.t_barrett);
  return mod_t64(h * P.two64_mod_t + l, P.t, P.t_barrett);
}

// centred binomial, eta = 21, of the low 42 bits of a draw
__device__ __forceinline__ int cbd21_of(uint64_t lo) {
  const uint64_t m21 = (1ull << 21) - 1;
  return __popcll(lo & m21) - __popcll((lo >> 21) & m21);
}

// Flooding term e1 = v - 2^F mod q for the 256-bit w[0] + w[1] 2^64 + ..,
// keeping its low F + 1 bits (v); Horner over the 64-bit words with
// qb = floor(2^64 / q), r64 = 2^64 mod q and two_f = 2^F mod q.
__device__ __forceinline__ uint64_t flood_e1(uint64_t (&w)[4], uint32_t F, uint64_t q, uint64_t qb,
                                             uint64_t r64, uint64_t r64s, uint64_t two_f) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int keep = (int)F + 1 - 64 * i;
    if (keep <= 0) w[i] = 0;
    else if (keep < 64) w[i] &= (1ull << keep) - 1;
  }
  uint64_t r = mod_t64(w[3], q, qb);
#pragma unroll
  for (int i = 2; i >= 0; --i) r = add_mod(mul_shoup(r, r64, r64s, q), mod_t64(w[i], q, qb), q);
  return sub_mod(r, two_f, q);
}

// (hi 2^64 + lo) mod q for any q < 2^63 (not on the hot path).
__device__ __forceinline__ uint64_t mod_q128(uint64_t lo, uint64_t hi, uint64_t q) {
  u128 v = ((u128)hi << 64) | lo;
  return (uint64_t)(v % q);
}

// ------------------------------------------------------------------------
// ChaCha20 block function, RFC 8439 Sec. 2.3.  key = (seed lo, seed hi, 0..),
// nonce = (purpose, object lo, object hi), counter = block index.  Block c/4
// yields the 128-bit draws of coefficients 4(c/4) .. 4(c/4)+3, draw u being
// words 4u..4u+3 read as lo = w0 | w1 << 32, hi = w2 | w3 << 32.
// ------------------------------------------------------------------------
__device__ __forceinline__ uint32_t rotl32(uint32_t x, int n) { return __funnelshift_l(x, x, n); }

#define SANNS_QR(a, b, c, d)             \
  a += b; d ^= a; d = rotl32(d, 16);     \
  c += d; b ^= c; b = rotl32(b, 12);     \
  a += b; d ^= a; d = rotl32(d, 8);      \
  c += d; b ^= c; b = rotl32(b, 7);

__device__ __forceinline__ void chacha20_block(uint64_t seed, uint32_t purpose, uint64_t object,
                                               uint32_t counter, uint32_t out[16]) {
  const uint32_t s0 = 0x61707865u, s1 = 0x3320646eu, s2 = 0x79622d32u, s3 = 0x6b206574u;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint32_t n0 = purpose, n1 = (uint32_t)object, n2 = (uint32_t)(object >> 32);
  uint32_t x0 = s0, x1 = s1, x2 = s2, x3 = s3;
  uint32_t x4 = k0, x5 = k1, x6 = 0, x7 = 0, x8 = 0, x9 = 0, x10 = 0, x11 = 0;
  uint32_t x12 = counter, x13 = n0, x14 = n1, x15 = n2;
#pragma unroll
  for (int r = 0; r < 10; r++) {
    SANNS_QR(x0, x4, x8, x12)
    SANNS_QR(x1, x5, x9, x13)
    SANNS_QR(x2, x6, x10, x14)
    SANNS_QR(x3, x7, x11, x15)
    SANNS_QR(x0, x5, x10, x15)
    SANNS_QR(x1, x6, x11, x12)
    SANNS_QR(x2, x7, x8, x13)
    SANNS_QR(x3, x4, x9, x14)
  }
  out[0] = x0 + s0;   out[1] = x1 + s1;   out[2] = x2 + s2;   out[3] = x3 + s3;
  out[4] = x4 + k0;   out[5] = x5 + k1;   out[6] = x6;        out[7] = x7;
  out[8] = x8;        out[9] = x9;        out[10] = x10;      out[11] = x11;
  out[12] = x12 + counter; out[13] = x13 + n0; out[14] = x14 + n1; out[15] = x15 + n2;
}
#undef SANNS_QR

__device__ __forceinline__ void draw_pair(const uint32_t blk[16], int u, uint64_t& lo,
                                          uint64_t& hi) {
  lo = (uint64_t)blk[4 * u] | ((uint64_t)blk[4 * u + 1] << 32);
  hi = (uint64_t)blk[4 * u + 2] | ((uint64_t)blk[4 * u + 3] << 32);
}

// ------------------------------------------------------------------------
// negacyclic NTT on a polynomial held in shared memory, executed by the whole
// block.  Forward: Cooley-Tukey with Harvey's lazy butterflies, values kept
// in [0, 4q); output slot s = a(psi^(2 brv(s) + 1)), canonicalised to [0, q).
// Inverse: Gentleman-Sande, values in [0, 2q), N^-1 folded at the end.
// Stages are grouped four at a time: a thread loads 16 elements that are
// closed under four consecutive stages, runs them in registers and writes
// back, so N = 8192 takes one radix-2 stage and three radix-16 passes.
// Callers synchronise the block before and after.
// ------------------------------------------------------------------------
// Shared-memory polynomials are stored padded, one spare word after every
// 16, so that the stride-16 accesses of the radix-16 passes hit distinct banks.
__host__ __device__ __forceinline__ uint32_t SP(uint32_t x) { return x + (x >> 4); }

// Storage format of the encoded database (values below 2^60): bits 0..29 in
// the low 32-bit word, bits 30..59 in the high word, so that the MAC reads
// the 30-bit halves it multiplies without splitting them.
__host__ __device__ __forceinline__ uint64_t split30(uint64_t y) {
  return (y & ((1ull << 30) - 1)) | ((y >> 30) << 32);
}
__host__ __device__ __forceinline__ uint64_t join30(uint64_t v) {
  return (v & 0xffffffffull) | ((v >> 32) << 30);
}
__host__ __device__ __forceinline__ uint32_t ntt_smem_words(uint32_t N) { return N + N / 16; }

// Global <-> padded shared-memory copies of one polynomial by the whole block,
// 16-byte accesses, eight in flight per thread before any is used.
__device__ __forceinline__ void load_poly(uint64_t* sa, const uint64_t* __restrict__ g, uint32_t N) {
  const uint32_t step = 2 * blockDim.x;
  for (uint32_t base = 0; base < N; base += 8 * step) {
    ulonglong2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint32_t x = base + r * step + 2 * threadIdx.x;
      v[r] = x < N ? __ldg(reinterpret_cast<const ulonglong2*>(g + x)) : make_ulonglong2(0, 0);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint32_t x = base + r * step + 2 * threadIdx.x;
      if (x < N) {
        sa[SP(x)] = v[r].x;
        sa[SP(x + 1)] = v[r].y;
      }
    }
  }
}

__device__ __forceinline__ void store_poly(uint64_t* __restrict__ g, const uint64_t* sa, uint32_t N) {
  for (uint32_t x = 2 * threadIdx.x; x < N; x += 2 * blockDim.x)
    *reinterpret_cast<ulonglong2*>(g + x) = make_ulonglong2(sa[SP(x)], sa[SP(x + 1)]);
}

__device__ __forceinline__ void fwd_bfly(uint64_t& X, uint64_t& Y, uint64_t w, uint64_t ws,
                                         uint64_t q, uint64_t q2) {
  X = csub(X, q2);
  const uint64_t T = mul_shoup_lazy(Y, w, ws, q);
  Y = X - T + q2;
  X = X + T;
}

__device__ __forceinline__ void inv_bfly(uint64_t& X, uint64_t& Y, uint64_t w, uint64_t ws,
                                         uint64_t q, uint64_t q2) {
  const uint64_t S = csub(X + Y, q2);
  const uint64_t D = X - Y + q2;
  X = S;
  Y = mul_shoup_lazy(D, w, ws, q);
}

// The same butterfly on values kept below 4q (q < 2^61, so sums stay below
// 2^64): bound = 4q.
__device__ __forceinline__ void inv_bfly4(uint64_t& X, uint64_t& Y, uint64_t w, uint64_t ws,
                                          uint64_t q, uint64_t q4) {
  const uint64_t S = csub(X + Y, q4);
  const uint64_t D = X - Y + q4;
  X = S;
  Y = mul_shoup_lazy4(D, w, ws, q);
}

template <bool LAZY4>
__device__ __forceinline__ void inv_bfly_t(uint64_t& X, uint64_t& Y, uint64_t w, uint64_t ws,
                                           uint64_t q, uint64_t bound) {
  if (LAZY4) inv_bfly4(X, Y, w, ws, q, bound);
  else inv_bfly(X, Y, w, ws, q, bound);
}

// first_st: leading radix-2 stages the caller has already done (values then
// lazily below 4q), at most logN & 3.
__device__ __forceinline__ void ntt_forward_smem(uint64_t* a, const PrimeSet& P, int j, uint32_t first_st = 0) {
  const uint32_t N = P.N, logN = P.logN;
  const uint64_t q = P.q[j], q2 = 2 * q;
  const ulonglong2* tw = P.tw + (size_t)j * N;
  const uint32_t r2 = logN & 3;  // leading radix-2 stages
  uint32_t lt = logN - 1 - first_st;  // log2 of the butterfly distance t
  for (uint32_t st = first_st; st < r2; ++st, --lt) {
    const uint32_t t = 1u << lt, m = 1u << st;
    for (uint32_t bf = threadIdx.x; bf < N / 2; bf += blockDim.x) {
      const uint32_t i = bf >> lt, x = (i << (lt + 1)) + (bf & (t - 1));
      uint64_t X = a[SP(x)], Y = a[SP(x + t)];
      const ulonglong2 w = __ldg(tw + m + i);
      fwd_bfly(X, Y, w.x, w.y, q, q2);
      a[SP(x)] = X;
      a[SP(x + t)] = Y;
    }
    __syncthreads();
  }
  // radix-16 passes: stages t, t/2, t/4, t/8 with t = 2^lt; a thread owns the
  // 16 elements x0 + k S (S = t/8) of one group; in stage s the lower element
  // k of a pair uses twiddle m_s + (g << s) + (k >> (4 - s)), m_s = N / (2 t_s)
  for (; lt >= 3 && lt + 1 <= logN; lt -= 4) {
    const uint32_t ls = lt - 3, S = 1u << ls;
    const uint32_t m0 = 1u << (logN - 1 - lt);
    for (uint32_t th = threadIdx.x; th < N / 16; th += blockDim.x) {
      const uint32_t g = th >> ls, b = th & (S - 1);
      const uint32_t x0 = (g << (lt + 1)) + b;
      uint64_t v[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = a[SP(x0 + (k << ls))];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int hk = 8 >> s;
        const uint32_t base = (m0 << s) + (g << s);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          if (k & hk) continue;
          const ulonglong2 w = __ldg(tw + base + (k >> (4 - s)));
          fwd_bfly(v[k], v[k + hk], w.x, w.y, q, q2);
        }
      }
      // values stay lazily below 4q between passes; the last pass (lt = 3)
      // stores them canonical
      if (lt == 3) {
#pragma unroll
        for (int k = 0; k < 16; ++k) a[SP(x0 + (k << ls))] = csub(csub(v[k], q2), q);
      } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) a[SP(x0 + (k << ls))] = v[k];
      }
    }
    __syncthreads();
    if (lt < 4) break;
  }
  if (r2 == logN) {  // N < 16: no radix-16 pass canonicalised the values
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) a[SP(x)] = csub(csub(a[SP(x)], q2), q);
  }
}

// One radix-16 pass of the inverse transform over the padded shared copy:
// stages t, 2t, 4t, 8t with t = 2^lt; a thread owns the 16 elements x0 + k t
// of one group; in stage s the lower element k of a pair uses twiddle
// h_s + (g << (3 - s)) + (k >> (s + 1)), h_s = N / (2 t 2^s).
// bound = 2q (values below 2q) or, with LAZY4, 4q (values below 4q).
template <bool LAZY4 = false>
__device__ __forceinline__ void inv_pass16(uint64_t* a, const ulonglong2* tw, uint32_t N,
                                           uint32_t logN, uint32_t lt, uint64_t q, uint64_t q2) {
  for (uint32_t th = threadIdx.x; th < N / 16; th += blockDim.x) {
    const uint32_t g = th >> lt, b = th & ((1u << lt) - 1);
    const uint32_t x0 = (g << (lt + 4)) + b;
    uint64_t v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = a[SP(x0 + (k << lt))];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int hk = 1 << s;
      const uint32_t base = (1u << (logN - 1 - lt - s)) + (g << (3 - s));
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (k & hk) continue;
        const ulonglong2 w = __ldg(tw + base + (k >> (s + 1)));
        inv_bfly_t<LAZY4>(v[k], v[k + hk], w.x, w.y, q, q2);
      }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) a[SP(x0 + (k << lt))] = v[k];
  }
}

// One radix-2 stage of the inverse transform, butterfly distance t = 2^lt.
template <bool LAZY4 = false>
__device__ __forceinline__ void inv_pass2(uint64_t* a, const ulonglong2* tw, uint32_t N,
                                          uint32_t logN, uint32_t lt, uint64_t q, uint64_t q2) {
  const uint32_t t = 1u << lt, h = 1u << (logN - 1 - lt);
  for (uint32_t bf = threadIdx.x; bf < N / 2; bf += blockDim.x) {
    const uint32_t i = bf >> lt, x = (i << (lt + 1)) + (bf & (t - 1));
    uint64_t X = a[SP(x)], Y = a[SP(x + t)];
    const ulonglong2 w = __ldg(tw + h + i);
    inv_bfly_t<LAZY4>(X, Y, w.x, w.y, q, q2);
    a[SP(x)] = X;
    a[SP(x + t)] = Y;
  }
}

__device__ __forceinline__ void ntt_inverse_smem(uint64_t* a, const PrimeSet& P, int j) {
  const uint32_t N = P.N, logN = P.logN;
  const uint64_t q = P.q[j], q2 = 2 * q;
  const ulonglong2* tw = P.itw + (size_t)j * N;
  const uint32_t passes = logN >> 2;
  const uint64_t ni = P.n_inv[j], nis = P.n_inv_shoup[j];
  uint32_t lt = 0;
  for (uint32_t ps = 0; ps < passes; ++ps, lt += 4) {
    inv_pass16(a, tw, N, logN, lt, q, q2);
    __syncthreads();
  }
  if (lt == logN) {
    // log2 N a multiple of 4: N^-1 in a pass of its own
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) a[SP(x)] = mul_shoup(a[SP(x)], ni, nis, q);
    return;
  }
  for (; lt + 1 < logN; ++lt) {
    inv_pass2(a, tw, N, logN, lt, q, q2);
    __syncthreads();
  }
  // the last stage (distance N/2, one twiddle psi^-brv(1)) with N^-1 folded
  // in: the sum side times N^-1, the difference side times psi^-brv(1) N^-1;
  // both canonical
  const uint64_t wl = P.last_inv[j], wls = P.last_inv_shoup[j];
  for (uint32_t x = threadIdx.x; x < N / 2; x += blockDim.x) {
    const uint64_t X = a[SP(x)], Y = a[SP(x + N / 2)];
    a[SP(x)] = mul_shoup(csub(X + Y, q2), ni, nis, q);
    a[SP(x + N / 2)] = mul_shoup(X - Y + q2, wl, wls, q);
  }
}

}  // namespace sanns
