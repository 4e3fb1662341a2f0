// Host-side derivation of the BFV/RNS constants: NTT-friendly primes, the
// primitive 2N-th roots, the plaintext modulus, Delta = floor(Q/t) mod q_j,
// CRT and Montgomery constants and the twiddle tables.  Sec. 7.1 of the paper
// fixes N = 2^13, a 180-bit q in three words and t = 2^b_d; the rest are the
// readings stated in sanns.h.
#include <cstring>
#include <string>

#include "internal.h"

namespace sanns {

namespace {

uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

uint64_t powmod(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  for (; e; e >>= 1) {
    if (e & 1) r = mulmod(r, a, m);
    a = mulmod(a, a, m);
  }
  return r;
}

// Deterministic Miller-Rabin for 64-bit n (bases = the first 12 primes).
bool is_prime_u64(uint64_t n) {
  static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (uint64_t p : bases)
    if (n % p == 0) return n == p;
  uint64_t d = n - 1;
  int r = 0;
  while ((d & 1) == 0) { d >>= 1; ++r; }
  for (uint64_t a : bases) {
    uint64_t x = powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < r; ++i) {
      x = mulmod(x, x, n);
      if (x == n - 1) { comp = false; break; }
    }
    if (comp) return false;
  }
  return true;
}

uint64_t inv_mod(uint64_t a, uint64_t m) {  // m prime
  return powmod(a, m - 2, m);
}

uint32_t bitrev(uint32_t x, uint32_t bits) {
  uint32_t r = 0;
  for (uint32_t b = 0; b < bits; ++b) { r = (r << 1) | (x & 1); x >>= 1; }
  return r;
}

}  // namespace

uint64_t shoup_of(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

uint64_t smallest_psi(uint64_t q, uint64_t N) {
  const uint64_t m = 2 * N;
  // psi0 of order exactly 2N, then the smallest of its odd powers
  uint64_t psi0 = 0;
  for (uint64_t g = 2;; ++g) {
    psi0 = powmod(g, (q - 1) / m, q);
    if (powmod(psi0, N, q) == q - 1) break;
  }
  uint64_t sq = mulmod(psi0, psi0, q), cur = psi0, best = psi0;
  for (uint64_t k = 1; k < N; ++k) {
    cur = mulmod(cur, sq, q);
    if (cur < best) best = cur;
  }
  return best;
}

int derive_params(const sanns_params& in, uint64_t q[], uint64_t psi[], uint64_t* t_out) {
  const uint64_t N = in.N, m = 2 * N;
  if (in.prime_bits < 20 || in.prime_bits > 60) return fail(SANNS_EINVAL, "prime_bits must be in [20, 60]");
  // largest x < 2^bits with x = 1 mod 2N, stepping down by 2N
  const uint64_t top = 1ull << in.prime_bits;
  uint64_t x = ((top - 1) / m) * m + 1;
  if (x >= top) x -= m;
  uint32_t found = 0;
  while (found < in.L) {
    if (x < m) return fail(SANNS_EINVAL, "not enough NTT-friendly primes below 2^prime_bits");
    if (is_prime_u64(x)) q[found++] = x;
    x -= m;
  }
  for (uint32_t j = 0; j < in.L; ++j) psi[j] = smallest_psi(q[j], N);
  uint64_t t;
  if (in.t_rule == 0) {
    t = ((1ull << 24) / m) * m + 1;
    if (t <= (1ull << 24)) t += m;
    while (!is_prime_u64(t)) t += m;
  } else if (in.t_rule == 1) {
    uint32_t lg = 0;
    while ((1u << lg) < in.d) ++lg;
    uint32_t bd = 2 * in.b_c + lg;
    if (bd > 31) return fail(SANNS_EINVAL, "t = 2^(2 b_c + ceil(log2 d)) exceeds 2^31");
    t = 1ull << bd;
  } else {
    return fail(SANNS_EINVAL, "t_rule must be 0 or 1");
  }
  for (uint32_t j = 0; j < in.L; ++j)
    if (t >= q[j]) return fail(SANNS_EINVAL, "plaintext modulus must be below every prime");
  *t_out = t;
  return SANNS_OK;
}

void fill_prime_constants(PrimeSet& P, const uint64_t q[], uint64_t t, uint32_t L) {
  P.L = L;
  P.t = t;
  P.t_barrett = (uint64_t)(((u128)1 << 64) / t);
  P.two64_mod_t = (uint64_t)(((u128)1 << 64) % t);
  // Q mod t, for Delta mod q_j = -(Q mod t) t^-1 (mod q_j), which follows from
  // Q - (Q mod t) = t Delta and Q = 0 mod q_j.
  uint64_t Q_mod_t = 1 % t;
  for (uint32_t j = 0; j < L; ++j) Q_mod_t = mulmod(Q_mod_t, q[j] % t, t);
  for (uint32_t j = 0; j < L; ++j) {
    const uint64_t qj = q[j];
    P.q[j] = qj;
    // -q^-1 mod 2^64 by Newton iteration (x <- x (2 - q x) doubles the bits)
    uint64_t inv = qj;  // correct to 3 bits for odd q
    for (int it = 0; it < 6; ++it) inv *= 2 - qj * inv;
    P.q_neg_inv[j] = (uint64_t)0 - inv;
    P.r64[j] = (uint64_t)(((u128)1 << 64) % qj);
    P.r64_shoup[j] = shoup_of(P.r64[j], qj);
    uint64_t tinv = inv_mod(t % qj, qj);
    uint64_t dl = mulmod((qj - Q_mod_t % qj) % qj, tinv, qj);
    P.delta[j] = dl;
    P.delta_shoup[j] = shoup_of(dl, qj);
    P.n_inv[j] = inv_mod(P.N % qj, qj);
    P.n_inv_shoup[j] = shoup_of(P.n_inv[j], qj);
    uint64_t qhat = 1 % qj;
    for (uint32_t i = 0; i < L; ++i)
      if (i != j) qhat = mulmod(qhat, q[i] % qj, qj);
    P.crt_inv[j] = inv_mod(qhat, qj);
    P.crt_inv_shoup[j] = shoup_of(P.crt_inv[j], qj);
  }
}

void fill_twiddles(uint32_t N, uint64_t q, uint64_t psi, uint64_t* tw, uint64_t* tws,
                   uint64_t* itw, uint64_t* itws) {
  uint32_t logN = 0;
  while ((1u << logN) < N) ++logN;
  // powers psi^e for e in [0, N) and psi^-e, then scatter by bit reversal
  const uint64_t psi_inv = inv_mod(psi, q);
  uint64_t p = 1, pi = 1;
  for (uint32_t e = 0; e < N; ++e) {
    uint32_t m = bitrev(e, logN);  // brv is an involution: brv(m) = e
    tw[m] = p;
    itw[m] = pi;
    p = mulmod(p, psi, q);
    pi = mulmod(pi, psi_inv, q);
  }
  for (uint32_t m = 0; m < N; ++m) {
    tws[m] = shoup_of(tw[m], q);
    itws[m] = shoup_of(itw[m], q);
  }
}

}  // namespace sanns
