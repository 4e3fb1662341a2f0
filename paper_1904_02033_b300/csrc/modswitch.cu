// Modulus switching of the response ciphertexts from Q = q_0 q_1 ... q_{L-1}
// down to q_0 (the standard BFV rescaling of [FV12]; SANNS sends its
// responses at the full modulus, so this is an option beyond the paper's
// protocol): every coefficient c in [0, Q) becomes round(q_0 c / Q) mod q_0,
// and the client decrypts modulo q_0.  The response then takes 1/L of the
// bytes on the wire.
//
// In RNS, with P = q_1 ... q_{L-1} (so q_0 c / Q = c / P) and
// delta = c mod P taken in (-P/2, P/2) (P is odd, so there is no tie),
//     round(c / P) = (c - delta) / P,
// and modulo q_0 that is (c_0 - delta) P^-1.  delta comes from the residues
// c_1 .. c_{L-1} through Garner's mixed-radix digits
//     delta = v_1 + q_1 v_2 + q_1 q_2 v_3 + ...,  0 <= v_m < q_m,
// its sign from comparing those digits with the digits of (P - 1) / 2 (most
// significant first), and its value mod q_0 from the digits times
// q_1 .. q_{m-1} mod q_0.  Primes are in descending order, so every digit
// and residue is below q_0.  No 128-bit arithmetic on the device.
#include "internal.h"

namespace sanns {

namespace {

uint64_t mulm(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

uint64_t powm(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  for (; e; e >>= 1) {
    if (e & 1) r = mulm(r, a, m);
    a = mulm(a, a, m);
  }
  return r;
}

// In place on [tuples][L][N]: coefficient x of tuple t is read from its L
// rows and round(q_0 c / Q) mod q_0 written over row 0.  One thread per
// (tuple, coefficient), coefficients fastest (coalesced rows).
__global__ void __launch_bounds__(256) mod_switch_kernel(PrimeSet P, ModSwitchConsts C,
                                                         uint64_t* __restrict__ buf, uint64_t total) {
  const uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (gid >= total) return;
  const uint32_t N = P.N, L = P.L;
  const uint64_t tup = gid >> P.logN, x = gid & (N - 1);
  uint64_t* row = buf + tup * L * N + x;
  uint64_t r[kMaxPrimes], v[kMaxPrimes];
#pragma unroll
  for (int j = 0; j < kMaxPrimes; ++j) r[j] = j < (int)L ? row[(uint64_t)j * N] : 0;
  // Garner digits of c mod P
  v[0] = 0;
  v[1] = r[1];
#pragma unroll
  for (int i = 2; i < kMaxPrimes; ++i) {
    if (i >= (int)L) break;
    const uint64_t qi = P.q[i];
    uint64_t s = 0;
#pragma unroll
    for (int m = 1; m < i; ++m) s = add_mod(s, mul_shoup(v[m], C.g[i][m], C.gs[i][m], qi), qi);
    v[i] = mul_shoup(sub_mod(r[i], s, qi), C.ginv[i], C.ginvs[i], qi);
  }
  // sign: delta > (P - 1) / 2, compared digit by digit from the top
  bool neg = false, decided = false;
#pragma unroll
  for (int m = kMaxPrimes - 1; m >= 1; --m) {
    if (m >= (int)L || decided) continue;
    if (v[m] != C.h[m]) {
      neg = v[m] > C.h[m];
      decided = true;
    }
  }
  const uint64_t q0 = P.q[0];
  uint64_t d0 = 0;
#pragma unroll
  for (int m = 1; m < kMaxPrimes; ++m)
    if (m < (int)L) d0 = add_mod(d0, mul_shoup(v[m], C.w0[m], C.w0s[m], q0), q0);
  if (neg) d0 = sub_mod(d0, C.p0, q0);
  row[0] = mul_shoup(sub_mod(r[0], d0, q0), C.pinv0, C.pinv0s, q0);
}

}  // namespace

void make_mod_switch_consts(const PrimeSet& P, ModSwitchConsts* C) {
  memset(C, 0, sizeof(*C));
  const uint32_t L = P.L;
  const uint64_t q0 = P.q[0];
  for (uint32_t i = 2; i < L; ++i) {
    const uint64_t qi = P.q[i];
    uint64_t prod = 1 % qi;                 // q_1 .. q_{m-1} mod q_i
    for (uint32_t m = 1; m < i; ++m) {
      C->g[i][m] = prod;
      C->gs[i][m] = shoup_of(prod, qi);
      prod = mulm(prod, P.q[m] % qi, qi);
    }
    C->ginv[i] = powm(prod, qi - 2, qi);    // (q_1 .. q_{i-1})^-1 mod q_i
    C->ginvs[i] = shoup_of(C->ginv[i], qi);
  }
  uint64_t prod0 = 1 % q0;                  // q_1 .. q_{m-1} mod q_0
  for (uint32_t m = 1; m < L; ++m) {
    C->w0[m] = prod0;
    C->w0s[m] = shoup_of(prod0, q0);
    prod0 = mulm(prod0, P.q[m] % q0, q0);
  }
  C->p0 = prod0;                            // P mod q_0
  C->pinv0 = L > 1 ? powm(prod0, q0 - 2, q0) : 1;
  C->pinv0s = shoup_of(C->pinv0, q0);
  // (P - 1) / 2 in the mixed radix: P - 1 has every digit q_m - 1; halve
  // from the most significant digit, carrying the remainder down
  uint64_t carry = 0;
  for (uint32_t m = L - 1; m >= 1; --m) {
    const u128 cur = (u128)(P.q[m] - 1) + (u128)carry * P.q[m];
    C->h[m] = (uint64_t)(cur / 2);
    carry = (uint64_t)(cur % 2);
  }
}

cudaError_t launch_mod_switch(const PrimeSet& P, const ModSwitchConsts& C, uint64_t* buf, uint64_t tuples,
                              cudaStream_t st) {
  if (P.L < 2 || tuples == 0) return cudaSuccess;
  const uint64_t total = tuples * P.N;
  mod_switch_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, C, buf, total);
  return cudaGetLastError();
}

}  // namespace sanns
