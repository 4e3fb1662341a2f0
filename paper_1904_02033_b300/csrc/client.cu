// Client-side kernels of Pi_ls (steps 1, 2 and 4): key generation, private-key
// BFV encryption of the query coordinates as constant plaintexts, and
// decryption of the masked distance ciphertexts with an exact RNS
// scale-and-round.
#include "internal.h"

namespace sanns {

namespace {

__host__ __device__ inline uint32_t blk_threads(uint32_t N) { return N / 16 < 32 ? 32 : (N / 16 > 256 ? 256 : N / 16); }

// One block per prime j: s is drawn by every block (cheap) and lifted mod q_j.
__global__ void __launch_bounds__(512) keygen_kernel(PrimeSet P, uint64_t seed, int8_t* s, uint64_t* s_hat,
                              uint64_t* s_hat_shoup) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N, j = blockIdx.x;
  const uint64_t q = P.q[j];
  for (uint32_t u = threadIdx.x; u < N / 4; u += blockDim.x) {
    uint32_t blk[16];
    chacha20_block(seed, kPurposeSk, 0, u, blk);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      uint64_t lo, hi;
      draw_pair(blk, v, lo, hi);
      int sv = (int)(lo % 3) - 1;
      sa[SP(4 * u + v)] = sv < 0 ? q - 1 : (uint64_t)sv;
      if (j == 0) s[4 * u + v] = (int8_t)sv;
    }
  }
  __syncthreads();
  ntt_forward_smem(sa, P, j);
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
    uint64_t v = sa[SP(x)];
    s_hat[(size_t)j * N + x] = v;
    s_hat_shoup[(size_t)j * N + x] = (uint64_t)(((u128)v << 64) / q);
  }
}

// One block per (i, j, b): NTT of the error polynomial of coordinate i, then
// c1 = a, c0 = -a s_hat + e_hat + Delta m slot by slot.
__global__ void __launch_bounds__(512) encrypt_kernel(PrimeSet P, const uint64_t* __restrict__ s_hat,
                               const uint64_t* __restrict__ s_hat_shoup,
                               const uint8_t* __restrict__ qv, uint32_t d, uint64_t seed,
                               const uint64_t* __restrict__ qids, uint64_t* __restrict__ ct) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N, L = P.L;
  const uint32_t i = blockIdx.x, j = blockIdx.y, b = blockIdx.z;
  const uint64_t q = P.q[j];
  const uint64_t qid = qids[b];
  const uint64_t e_obj = (qid << 16) | i;
  for (uint32_t u = threadIdx.x; u < N / 4; u += blockDim.x) {
    uint32_t blk[16];
    chacha20_block(seed, kPurposeE, e_obj, u, blk);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      uint64_t lo, hi;
      draw_pair(blk, v, lo, hi);
      const uint64_t m21 = (1ull << 21) - 1;
      int e = __popcll(lo & m21) - __popcll((lo >> 21) & m21);
      sa[SP(4 * u + v)] = e < 0 ? q - (uint64_t)(-e) : (uint64_t)e;
    }
  }
  __syncthreads();
  ntt_forward_smem(sa, P, j);
  __syncthreads();
  const uint64_t t = P.t;
  const uint64_t m = (t - (2ull * qv[(size_t)b * d + i]) % t) % t;
  const uint64_t dm = mul_shoup(m, P.delta[j], P.delta_shoup[j], q);
  const uint64_t a_obj = (qid << 16) | ((uint64_t)j << 12) | i;
  uint64_t* c0 = ct + ((((size_t)b * d + i) * 2 + 0) * L + j) * N;
  uint64_t* c1 = ct + ((((size_t)b * d + i) * 2 + 1) * L + j) * N;
  const uint64_t* sh = s_hat + (size_t)j * N;
  const uint64_t* shs = s_hat_shoup + (size_t)j * N;
  for (uint32_t u = threadIdx.x; u < N / 4; u += blockDim.x) {
    uint32_t blk[16];
    chacha20_block(seed, kPurposeA, a_obj, u, blk);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      uint64_t lo, hi;
      draw_pair(blk, v, lo, hi);
      const uint32_t s = 4 * u + v;
      const uint64_t a = mod_q128(lo, hi, q);
      const uint64_t as = mul_shoup(a, sh[s], shs[s], q);
      uint64_t v0 = sub_mod(sa[SP(s)], as, q);
      v0 = add_mod(v0, dm, q);
      c1[s] = a;
      c0[s] = v0;
    }
  }
}

// Seeded query ciphertexts: the server rebuilds c1 = a from the same stream
// as encrypt_kernel and places the received c0 beside it.  One block per
// (i, j, b); c0_in is [B][d][L][N], ct is [B][d][2][L][N].
__global__ void __launch_bounds__(256) seeded_query_kernel(PrimeSet P, const uint64_t* __restrict__ c0_in,
                                                           uint32_t d, uint64_t seed,
                                                           const uint64_t* __restrict__ qids,
                                                           uint64_t* __restrict__ ct) {
  const uint32_t N = P.N, L = P.L;
  const uint32_t i = blockIdx.x, j = blockIdx.y, b = blockIdx.z;
  const uint64_t q = P.q[j];
  const uint64_t a_obj = (qids[b] << 16) | ((uint64_t)j << 12) | i;
  const uint64_t* src = c0_in + (((size_t)b * d + i) * L + j) * N;
  uint64_t* c0 = ct + ((((size_t)b * d + i) * 2 + 0) * L + j) * N;
  uint64_t* c1 = ct + ((((size_t)b * d + i) * 2 + 1) * L + j) * N;
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) c0[x] = src[x];
  for (uint32_t u = threadIdx.x; u < N / 4; u += blockDim.x) {
    uint32_t blk[16];
    chacha20_block(seed, kPurposeA, a_obj, u, blk);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      uint64_t lo, hi;
      draw_pair(blk, v, lo, hi);
      c1[4 * u + v] = mod_q128(lo, hi, q);
    }
  }
}

// Decryption, first half: one block per (b, k, j): v = c0 + INTT(NTT(c1) s_hat)
// for coefficient-form responses, v = INTT(c0 + c1 s_hat) for NTT-form ones.
__global__ void __launch_bounds__(512) decrypt_phase_kernel(PrimeSet P, const uint64_t* __restrict__ ct_out,
                                     const uint64_t* __restrict__ s_hat,
                                     const uint64_t* __restrict__ s_hat_shoup, uint64_t K,
                                     uint64_t* __restrict__ v, int ntt_form) {
  extern __shared__ uint64_t sa[];
  const uint32_t N = P.N, L = P.L;
  const uint64_t idx = blockIdx.x;  // (b K + k) L + j
  const uint32_t j = (uint32_t)(idx % L);
  const uint64_t bk = idx / L;
  const uint64_t q = P.q[j];
  const uint64_t* c0 = ct_out + ((bk * 2 + 0) * L + j) * N;
  const uint64_t* c1 = ct_out + ((bk * 2 + 1) * L + j) * N;
  if (ntt_form) {
    const uint64_t* sh = s_hat + (size_t)j * N;
    const uint64_t* shs = s_hat_shoup + (size_t)j * N;
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x)
      sa[SP(x)] = add_mod(mul_shoup(c1[x], sh[x], shs[x], q), c0[x], q);
    __syncthreads();
    ntt_inverse_smem(sa, P, j);
    __syncthreads();
    uint64_t* o = v + idx * N;
    for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) o[x] = sa[SP(x)];
    return;
  }
  load_poly(sa, c1, N);
  __syncthreads();
  ntt_forward_smem(sa, P, j);
  __syncthreads();
  const uint64_t* sh = s_hat + (size_t)j * N;
  const uint64_t* shs = s_hat_shoup + (size_t)j * N;
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) sa[SP(x)] = mul_shoup(sa[SP(x)], sh[x], shs[x], q);
  __syncthreads();
  ntt_inverse_smem(sa, P, j);
  __syncthreads();
  uint64_t* o = v + idx * N;
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) o[x] = add_mod(sa[SP(x)], c0[x], q);
}

// Decryption, second half, one thread per (b, pos):
//   t w / Q = sum_j x_j t / q_j - t alpha,  x_j = v_j (Q/q_j)^-1 mod q_j,
// with alpha an integer; mod t only the sum matters.  Writing x_j t =
// I_j q_j + R_j, m = (sum I_j + round(sum R_j / q_j)) mod t.  The fractions
// R_j / q_j are summed in 64.64 fixed point with an error below L 2^-64.  For
// a ciphertext with noise e, t w / Q = m - (Q mod t) m / Q + t e / Q, so the
// fraction lies within t (|e| + t) / Q of an integer -- far from 1/2 whenever
// decryption is correct at all -- and the truncation cannot change the
// rounding.
// With slot encoding (slots != 0) every coefficient of every block is
// decoded (n is then K N) and m is written over v[b][k][0][x], which only this
// thread reads; slot_decode_kernel takes it from there.
__global__ void scale_round_kernel(PrimeSet P, uint64_t* __restrict__ v, uint64_t K,
                                   uint64_t n, uint32_t B, const uint8_t* __restrict__ qv,
                                   uint32_t d, uint32_t* __restrict__ cli_share, int slots) {
  const uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (gid >= (uint64_t)B * n) return;
  const uint64_t b = gid / n, pos = gid % n;
  const uint32_t N = P.N, L = P.L;
  const uint64_t k = pos / N, x = pos % N;
  const uint64_t t = P.t;
  uint64_t isum = 0;   // mod t
  u128 fsum = 0;       // 64.64 fixed point
  for (uint32_t j = 0; j < L; ++j) {
    const uint64_t q = P.q[j];
    const uint64_t vj = v[((b * K + k) * L + j) * N + x];
    const uint64_t xj = mul_shoup(vj, P.crt_inv[j], P.crt_inv_shoup[j], q);
    const u128 prod = (u128)xj * t;
    const uint64_t I = (uint64_t)(prod / q);
    const uint64_t R = (uint64_t)(prod - (u128)I * q);
    isum = (isum + I % t) % t;
    fsum += ((u128)R << 64) / q;
  }
  const uint64_t whole = (uint64_t)(fsum >> 64);
  const uint64_t frac = (uint64_t)fsum;
  uint64_t m = (isum + whole + (frac >> 63)) % t;
  if (slots) {
    v[((b * K + k) * L + 0) * N + x] = m;
    return;
  }
  uint32_t qn = 0;
  const uint8_t* qq = qv + b * d;
  for (uint32_t i = 0; i < d; ++i) qn += (uint32_t)qq[i] * qq[i];
  cli_share[gid] = (uint32_t)((m + qn) % t);
}

// Slot encoding, the client's shares: one block per (b, k), the slots of the
// decrypted plaintext m (NTT_t of its coefficients) plus ||q||^2.
__global__ void __launch_bounds__(512) slot_decode_kernel(PrimeSet P, PrimeSet PT,
                                                          const uint64_t* __restrict__ v, uint64_t K,
                                                          uint64_t n, const uint8_t* __restrict__ qv,
                                                          uint32_t d, uint32_t* __restrict__ cli_share) {
  extern __shared__ uint64_t sa[];
  __shared__ uint32_t qn;
  const uint32_t N = P.N, L = P.L;
  const uint64_t bk = blockIdx.x, b = bk / K, k = bk % K;
  const uint64_t* m = v + (bk * L + 0) * N;
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) sa[SP(x)] = m[x];
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (uint32_t i = 0; i < d; ++i) acc += (uint32_t)qv[b * d + i] * qv[b * d + i];
    qn = acc;
  }
  __syncthreads();
  ntt_forward_smem(sa, PT, 0);
  __syncthreads();
  const uint64_t t = P.t;
  for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
    const uint64_t pos = k * N + x;
    if (pos >= n) break;
    cli_share[b * n + pos] = (uint32_t)((sa[SP(x)] + qn) % t);
  }
}

}  // namespace

cudaError_t launch_keygen(const PrimeSet& P, uint64_t seed, int8_t* s, uint64_t* s_hat,
                          uint64_t* s_hat_shoup, cudaStream_t st) {
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  cudaError_t e = cudaFuncSetAttribute(keygen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  keygen_kernel<<<P.L, blk_threads(P.N), smem, st>>>(P, seed, s, s_hat, s_hat_shoup);
  return cudaGetLastError();
}

cudaError_t launch_encrypt(const PrimeSet& P, const uint64_t* s_hat, const uint64_t* s_hat_shoup,
                           const uint8_t* qv, uint32_t B, uint32_t d, uint64_t seed,
                           const uint64_t* qids, uint64_t* ct, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  cudaError_t e = cudaFuncSetAttribute(encrypt_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(d, P.L, B);
  encrypt_kernel<<<grid, blk_threads(P.N), smem, st>>>(P, s_hat, s_hat_shoup, qv, d, seed, qids,
                                                       ct);
  return cudaGetLastError();
}

cudaError_t launch_seeded_query(const PrimeSet& P, const uint64_t* c0, uint32_t B, uint32_t d,
                                uint64_t seed, const uint64_t* qids, uint64_t* ct, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  dim3 grid(d, P.L, B);
  seeded_query_kernel<<<grid, 256, 0, st>>>(P, c0, d, seed, qids, ct);
  return cudaGetLastError();
}

cudaError_t launch_decrypt(const PrimeSet& P, const uint64_t* ct_out, const int8_t* s,
                           const uint64_t* s_hat, const uint64_t* s_hat_shoup, uint32_t B,
                           uint64_t K, uint64_t n, const uint8_t* qv, uint32_t d,
                           uint64_t* scratch, uint32_t* cli_share, bool ntt_form, const PrimeSet* PT,
                           cudaStream_t st) {
  (void)s;
  if (B == 0 || n == 0) return cudaSuccess;
  const size_t smem = sizeof(uint64_t) * ntt_smem_words(P.N);
  cudaError_t e = cudaFuncSetAttribute(decrypt_phase_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  decrypt_phase_kernel<<<(unsigned)((uint64_t)B * K * P.L), blk_threads(P.N), smem, st>>>(
      P, ct_out, s_hat, s_hat_shoup, K, scratch, ntt_form ? 1 : 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!PT) {
    const uint64_t total = (uint64_t)B * n;
    scale_round_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, scratch, K, n, B, qv, d,
                                                                        cli_share, 0);
    return cudaGetLastError();
  }
  const uint64_t total = (uint64_t)B * K * P.N;
  scale_round_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, scratch, K, K * P.N, B, qv, d,
                                                                      cli_share, 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(slot_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  slot_decode_kernel<<<(unsigned)((uint64_t)B * K), blk_threads(P.N), smem, st>>>(P, *PT, scratch, K, n, qv, d,
                                                                                   cli_share);
  return cudaGetLastError();
}

}  // namespace sanns
