// Circuit privacy of the distance responses.  The paper requires the AHE
// scheme to be circuit private and obtains it by noise flooding (Sec. 2.3,
// "Additive Homomorphic Encryption"; 108 bits of statistical circuit privacy
// with its parameters, Sec. 7.1).  With private-key BFV the server cannot
// re-randomise c1 = sum_i a_i g_i by itself, so the client publishes a public
// key pk = (-a s + e, a) and the server adds a fresh encryption of zero,
// (pk0 u + e1, pk1 u + e2), to every response block; e1 is the flooding term,
// uniform in [-2^F, 2^F).  Every draw is a counter-based ChaCha20 stream at
// the global database position, so the result is deterministic.
//   client:  public_key_kernel
//   server:  rerandomize_kernel (NTT domain, before the inverse transform)
//            flood_kernel       (coefficient domain, after it)
#include "internal.h"

namespace sanns {

namespace {

__host__ __device__ inline uint32_t pv_threads(uint32_t N) { return N / 16 < 32 ? 32 : (N / 16 > 256 ? 256 : N / 16); }

// One block per prime j: e (centred binomial, stream (seed, E_PK, 0)) lifted
// and transformed; a uniform mod q_j drawn in NTT form from (seed, A_PK, j);
// pk1 = a, pk0 = -a s_hat + e_hat slot by slot; layout pk[c][j][s].
__global__ void __launch_bounds__(256) public_key_kernel(PrimeSet P, const uint64_t* __restrict__ s_hat,
                                                         const uint64_t* __restrict__ s_hat_shoup,
                                                         uint64_t seed, uint64_t* __restrict__ pk) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N, L = P.L, j = blockIdx.x;
  const uint64_t q = P.q[j];
  for (uint32_t u = threadIdx.x; u < N / 4; u += blockDim.x) {
    uint32_t blk[16];
    chacha20_block(seed, kPurposeEPk, 0, u, blk);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      uint64_t lo, hi;
      draw_pair(blk, v, lo, hi);
      const int e = cbd21_of(lo);
      sa[SP(4 * u + v)] = e < 0 ? q - (uint64_t)(-e) : (uint64_t)e;
    }
  }
  __syncthreads();
  ntt_forward_smem(sa, P, j);
  __syncthreads();
  const uint64_t* sh = s_hat + (size_t)j * N;
  const uint64_t* shs = s_hat_shoup + (size_t)j * N;
  uint64_t* p0 = pk + (size_t)j * N;
  uint64_t* p1 = pk + ((size_t)L + j) * N;
  for (uint32_t u = threadIdx.x; u < N / 4; u += blockDim.x) {
    uint32_t blk[16];
    chacha20_block(seed, kPurposeAPk, j, u, blk);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      uint64_t lo, hi;
      draw_pair(blk, v, lo, hi);
      const uint32_t s = 4 * u + v;
      const uint64_t a = mod_q128(lo, hi, q);
      p1[s] = a;
      p0[s] = add_mod(sub_mod(0, mul_shoup(a, sh[s], shs[s], q), q), sa[SP(s)], q);
    }
  }
}

// Shoup companions floor(w 2^64 / q_j) of a [2][L][N] key (setup only).
__global__ void key_shoup_kernel(PrimeSet P, const uint64_t* __restrict__ pk, uint64_t* __restrict__ pks) {
  const uint64_t total = 2ull * P.L * P.N;
  const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (e >= total) return;
  const uint32_t j = (uint32_t)((e / P.N) % P.L);
  const uint64_t q = P.q[j], w = pk[e];
  pks[e] = (uint64_t)(((u128)w << 64) / q);
}

// One block per (b, k, j) of ct [B][K][2][L][N] (NTT form, in place): u
// ternary, (lo mod 3) - 1 of the draw (seed, U, qid_b) at global position
// pos0 + k N + x, transformed; then c += pk_c * u_hat for c = 0, 1.
__global__ void __launch_bounds__(256, 3) rerandomize_kernel(PrimeSet P, uint64_t* __restrict__ ct, uint64_t K,
                                                             uint64_t pos0, uint64_t seed,
                                                             const uint64_t* __restrict__ qids,
                                                             const uint64_t* __restrict__ pk,
                                                             const uint64_t* __restrict__ pks) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N, L = P.L;
  const uint64_t idx = blockIdx.x;  // (b K + k) L + j
  const uint32_t j = (uint32_t)(idx % L);
  const uint64_t bk = idx / L, k = bk % K, b = bk / K;
  const uint64_t q = P.q[j];
  const uint64_t g0 = pos0 + k * N;  // a multiple of N, hence of 4
  for (uint32_t u = threadIdx.x; u < N / 4; u += blockDim.x) {
    uint32_t blk[16];
    chacha20_block(seed, kPurposeU, qids[b], (uint32_t)(g0 / 4 + u), blk);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      uint64_t lo, hi;
      draw_pair(blk, v, lo, hi);
      const int uv = (int)(lo % 3) - 1;
      sa[SP(4 * u + v)] = uv < 0 ? q - 1 : (uint64_t)uv;
    }
  }
  __syncthreads();
  ntt_forward_smem(sa, P, j);
  __syncthreads();
  uint64_t* c0 = ct + ((bk * 2 + 0) * L + j) * N;
  uint64_t* c1 = ct + ((bk * 2 + 1) * L + j) * N;
  const uint64_t* p0 = pk + (size_t)j * N;
  const uint64_t* p1 = pk + ((size_t)L + j) * N;
  const uint64_t* s0 = pks + (size_t)j * N;
  const uint64_t* s1 = pks + ((size_t)L + j) * N;
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
    const uint64_t uh = sa[SP(x)];
    c0[x] = add_mod(c0[x], mul_shoup(uh, p0[x], s0[x], q), q);
    c1[x] = add_mod(c1[x], mul_shoup(uh, p1[x], s1[x], q), q);
  }
}

// One thread per four consecutive positions of one (b, k) (coefficient form,
// in place, every prime): e1 = v - 2^F with v the low F + 1 bits of
// lo_a + hi_a 2^64 + lo_b 2^128 + hi_b 2^192 (draws (seed, FLOOD_LO, qid) and
// (seed, FLOOD_HI, qid)), e2 = centred binomial of the draw (seed, E2, qid);
// c0 += e1 mod q_j, c1 += e2 mod q_j.
__global__ void flood_kernel(PrimeSet P, uint64_t* __restrict__ ct, uint32_t B, uint64_t K, uint64_t pos0,
                             uint64_t seed, const uint64_t* __restrict__ qids, uint32_t F,
                             PrivacyConsts C) {
  const uint32_t N = P.N, L = P.L;
  const uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t groups = (uint64_t)B * K * (N / 4);
  if (gid >= groups) return;
  const uint32_t x0 = (uint32_t)(gid % (N / 4)) * 4;
  const uint64_t bk = gid / (N / 4), k = bk % K, b = bk / K;
  const uint32_t ctr = (uint32_t)((pos0 + k * N + x0) / 4);
  const uint64_t qid = qids[b];
  uint32_t ba[16], bb[16], be[16];
  chacha20_block(seed, kPurposeFloodLo, qid, ctr, ba);
  chacha20_block(seed, kPurposeFloodHi, qid, ctr, bb);
  chacha20_block(seed, kPurposeE2, qid, ctr, be);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    uint64_t w[4], lo, hi;
    draw_pair(ba, v, w[0], w[1]);
    draw_pair(bb, v, w[2], w[3]);
    draw_pair(be, v, lo, hi);
    const int e2 = cbd21_of(lo);
    const uint32_t x = x0 + v;
    for (uint32_t j = 0; j < L; ++j) {
      const uint64_t q = P.q[j];
      uint64_t wj[4] = {w[0], w[1], w[2], w[3]};
      const uint64_t e1 = flood_e1(wj, F, q, C.q_barrett[j], P.r64[j], P.r64_shoup[j], C.two_f[j]);
      uint64_t* c0 = ct + ((bk * 2 + 0) * L + j) * N + x;
      uint64_t* c1 = ct + ((bk * 2 + 1) * L + j) * N + x;
      *c0 = add_mod(*c0, e1, q);
      *c1 = add_mod(*c1, e2 < 0 ? q - (uint64_t)(-e2) : (uint64_t)e2, q);
    }
  }
}

}  // namespace

cudaError_t launch_public_key(const PrimeSet& P, const uint64_t* s_hat, const uint64_t* s_hat_shoup,
                              uint64_t seed, uint64_t* pk, cudaStream_t st) {
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  cudaError_t e = cudaFuncSetAttribute(public_key_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  public_key_kernel<<<P.L, pv_threads(P.N), smem, st>>>(P, s_hat, s_hat_shoup, seed, pk);
  return cudaGetLastError();
}

cudaError_t launch_key_shoup(const PrimeSet& P, const uint64_t* pk, uint64_t* pks, cudaStream_t st) {
  const uint64_t total = 2ull * P.L * P.N;
  key_shoup_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, pk, pks);
  return cudaGetLastError();
}

cudaError_t launch_rerandomize(const PrimeSet& P, uint64_t* ct, uint32_t B, uint64_t K, uint64_t pos0,
                               uint64_t seed, const uint64_t* qids, const uint64_t* pk,
                               const uint64_t* pks, cudaStream_t st) {
  const uint64_t blocks = (uint64_t)B * K * P.L;
  if (blocks == 0) return cudaSuccess;
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  cudaError_t e = ensure_smem_attr((const void*)rerandomize_kernel, smem);
  if (e != cudaSuccess) return e;
  rerandomize_kernel<<<(unsigned)blocks, pv_threads(P.N), smem, st>>>(P, ct, K, pos0, seed, qids, pk, pks);
  return cudaGetLastError();
}

cudaError_t launch_flood(const PrimeSet& P, uint64_t* ct, uint32_t B, uint64_t K, uint64_t pos0,
                         uint64_t seed, const uint64_t* qids, uint32_t F, const PrivacyConsts& C,
                         cudaStream_t st) {
  const uint64_t groups = (uint64_t)B * K * (P.N / 4);
  if (groups == 0) return cudaSuccess;
  flood_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(P, ct, B, K, pos0, seed, qids, F, C);
  return cudaGetLastError();
}

}  // namespace sanns
