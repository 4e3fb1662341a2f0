"""BFV parameter derivation with exact Python integers.

TEST INFRASTRUCTURE ONLY (the oracle): only tests/, __graft_entry__.smoke()
and bench.py's cpu_baseline and reference legs may import this package.

The paper fixes N = 2^13 and a 180-bit ciphertext modulus made of three
machine words (Sec. 7.1, "Parameters") and a plaintext modulus t = 2^b_d with
b_d = 2 b_c + ceil(log2 d) (Fig. "hyperparameters": b_d, t).  It does not list
the primes or the root of unity (SEAL defaults).  Readings used here:

* primes: the L largest primes below 2^prime_bits with q = 1 (mod 2N);
* psi_j: the smallest primitive 2N-th root of unity mod q_j;
* t: rule 0 = the smallest prime above 2^24 with t = 1 (mod 2N); rule 1 = the
  paper's 2^(2 b_c + ceil(log2 d)) with b_c = 8;
* Delta = floor(Q / t), Q = prod q_j.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from functools import reduce

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (the first 12 prime bases)."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(N: int, L: int, bits: int) -> list[int]:
    """The L largest primes q < 2^bits with q = 1 (mod 2N), descending."""
    m = 2 * N
    x = ((2 ** bits - 1) // m) * m + 1
    if x >= 2 ** bits:
        x -= m
    out = []
    while len(out) < L:
        if x < 2:
            raise ValueError("not enough NTT primes")
        if is_prime(x):
            out.append(x)
        x -= m
    return out


def min_primitive_root_2n(q: int, N: int) -> int:
    """Smallest psi with psi^N = -1 (mod q), i.e. of multiplicative order 2N."""
    m = 2 * N
    assert (q - 1) % m == 0
    g = 2
    while True:
        psi0 = pow(g, (q - 1) // m, q)
        if pow(psi0, N, q) == q - 1:
            break
        g += 1
    # every primitive 2N-th root is psi0^k for odd k
    return min(pow(psi0, k, q) for k in range(1, m, 2))


def plain_modulus(N: int, rule: int, d: int, b_c: int = 8) -> int:
    """rule 0: smallest prime > 2^24 with t = 1 (mod 2N); rule 1: the paper's
    t = 2^b_d, b_d = 2 b_c + ceil(log2 d) (Fig. "hyperparameters")."""
    if rule == 0:
        m = 2 * N
        x = (2 ** 24 // m) * m + 1
        if x <= 2 ** 24:
            x += m
        while not is_prime(x):
            x += m
        return x
    if rule == 1:
        return 2 ** (2 * b_c + (d - 1).bit_length())
    raise ValueError("t_rule must be 0 or 1")


@dataclass
class Params:
    N: int
    L: int
    prime_bits: int
    t_rule: int
    d: int
    q: list[int] = field(default_factory=list)
    psi: list[int] = field(default_factory=list)
    t: int = 0
    Q: int = 0
    delta: int = 0

    @property
    def delta_mod_q(self) -> list[int]:
        """Delta = floor(Q / t) (BFV, Sec. 2.3) reduced mod each q_j."""
        return [self.delta % qj for qj in self.q]


def make_params(N: int, L: int, prime_bits: int, t_rule: int, d: int, b_c: int = 8) -> Params:
    """The BFV parameters of Sec. 7.1 ("Parameters": N, a three-word q, t) as
    exact integers: the L largest primes below 2^prime_bits that are 1 mod 2N,
    the smallest primitive 2N-th root psi of each, t by its rule (b_c bits
    per coordinate for the paper's rule), and Delta = floor(Q / t)."""
    if N & (N - 1) or N < 2:
        raise ValueError("N must be a power of two")
    q = ntt_primes(N, L, prime_bits)
    psi = [min_primitive_root_2n(qj, N) for qj in q]
    t = plain_modulus(N, t_rule, d, b_c)
    Q = reduce(lambda a, b: a * b, q, 1)
    return Params(N=N, L=L, prime_bits=prime_bits, t_rule=t_rule, d=d,
                  q=q, psi=psi, t=t, Q=Q, delta=Q // t)
