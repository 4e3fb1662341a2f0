"""CPU oracle for the encrypted query-point distance path of SANNS
(arxiv 1904.02033, Sec. 5.3 and Fig. "SANNS linear-scan protocol").

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import, call, link or run
anything in this package.  It shares no code with the CUDA library and never
imports it; the only thing both sides consume in common is the seeded input
generator module (paper_1904_02033_b300.inputs), which holds none of the
method's arithmetic.

Contents
  sanns_oracle.c  plain C loops: textbook NTT/INTT, ChaCha20 (RFC 8439),
                  keygen, encrypt, DB encoding, ct x pt MAC, INTT + mask,
                  the c0 + c1 s step of decryption, schoolbook products.
  params.py       exact-integer parameter derivation (primes, psi, t, Delta).
  bfv.py          ctypes wrappers + exact big-integer CRT scale-and-round;
                  circuit privacy (public key, re-randomisation, flooding);
                  slot encoding (the negacyclic transform mod t, slot shares).
  select.py       Algorithms 1 and 2 (NaiveTopk, ApproxTopk) in plaintext.
  clustering.py   Algorithm 4 (ClusteringKNNS) in plaintext on a given server
                  layout (groups of clusters with shuffled centres, stash).

Parity pins: every function above is pinned by a -m "not gpu" test against
something other than itself (O(N^2) NTT definition, schoolbook products,
RFC 8439 test vectors, decrypt(encrypt(m)) = m, brute-force distances,
sympy primality, closed forms for ApproxTopk, the mod-t transform as a ring
isomorphism, Algorithm 4 reducing to brute force when every cluster is
retrieved).  The concrete ciphertext bits depend on conventions the paper
leaves open (RNG layout, NTT order), so the paper prints none; encryption,
the response blocks, circuit privacy and decryption are each re-derived at
N = 64 from their definitions with schoolbook products and exact integers.
"""
from .bfv import Oracle, chacha20_block  # noqa: F401
from .params import make_params  # noqa: F401
