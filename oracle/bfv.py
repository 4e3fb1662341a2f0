"""The oracle's protocol steps: ctypes calls into the plain C loops plus the
exact big-integer CRT decryption.

TEST INFRASTRUCTURE ONLY (the oracle): only tests/, __graft_entry__.smoke()
and bench.py's cpu_baseline and reference legs may import this module.  It never imports the
CUDA package.

Follows SANNS (arxiv 1904.02033) Sec. 5.3 and Fig. "SANNS linear-scan
protocol" (Pi_ls) steps 1-4; BFV as in Sec. 2.3 [FV12].
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build
from .params import Params, make_params, min_primitive_root_2n

_lib = None


def lib():
    """The oracle's compiled C loops (built on first use)."""
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        u64p = C.POINTER(C.c_uint64)
        _lib.oracle_ntt_tables.argtypes = [C.c_uint32, C.c_uint64, C.c_uint64, u64p, u64p]
        _lib.oracle_ntt.argtypes = [u64p, C.c_uint32, C.c_uint64, u64p]
        _lib.oracle_intt.argtypes = [u64p, C.c_uint32, C.c_uint64, u64p]
        _lib.oracle_chacha20_block.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p]
        _lib.oracle_draw128.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint64, C.c_void_p]
        _lib.oracle_keygen.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]
        _lib.oracle_encrypt.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                                        C.c_uint64, C.c_void_p]
        _lib.oracle_encode_db.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                                          C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p]
        _lib.oracle_mac.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p]
        _lib.oracle_intt_mask.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                                          C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64,
                                          C.c_void_p, C.c_void_p]
        _lib.oracle_decrypt_phase.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                                              C.c_void_p]
        _lib.oracle_negacyclic_schoolbook.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32,
                                                      C.c_uint64, C.c_void_p]
        _lib.oracle_public_key.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p]
        _lib.oracle_rerandomize.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                                            C.c_uint64, C.c_uint64, C.c_uint64]
        _lib.oracle_flood.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64,
                                      C.c_uint64, C.c_uint64, C.c_uint32]
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


class _CParams(C.Structure):
    _fields_ = [("N", C.c_uint32), ("L", C.c_uint32), ("d", C.c_uint32), ("pad", C.c_uint32),
                ("t", C.c_uint64), ("q", C.c_void_p), ("fwd", C.c_void_p), ("inv", C.c_void_p),
                ("delta", C.c_void_p)]


class Oracle:
    """One BFV parameter set with its twiddle tables, for the C loops."""

    def __init__(self, N: int, L: int, prime_bits: int, t_rule: int, d: int, b_c: int = 8):
        self.P: Params = make_params(N, L, prime_bits, t_rule, d, b_c)
        self.b_c = b_c
        P = self.P
        self.N, self.L, self.d, self.t = N, L, d, P.t
        self.q = np.array(P.q, dtype=np.uint64)
        self.delta = np.array(P.delta_mod_q, dtype=np.uint64)
        self.fwd = np.zeros((L, N), dtype=np.uint64)
        self.inv = np.zeros((L, N), dtype=np.uint64)
        for j in range(L):
            f = self.fwd[j]
            v = self.inv[j]
            lib().oracle_ntt_tables(N, int(self.q[j]), P.psi[j],
                                    f.ctypes.data_as(C.POINTER(C.c_uint64)),
                                    v.ctypes.data_as(C.POINTER(C.c_uint64)))
        self._c = _CParams(N, L, d, 0, P.t, _p(self.q).value, _p(self.fwd).value,
                           _p(self.inv).value, _p(self.delta).value)
        # slot encoding: the negacyclic transform mod t (t = 1 mod 2N)
        self.slots_ok = (P.t - 1) % (2 * N) == 0
        if self.slots_ok:
            self.psi_t = min_primitive_root_2n(P.t, N)
            self.fwd_t = np.zeros(N, dtype=np.uint64)
            self.inv_t = np.zeros(N, dtype=np.uint64)
            lib().oracle_ntt_tables(N, P.t, self.psi_t,
                                    self.fwd_t.ctypes.data_as(C.POINTER(C.c_uint64)),
                                    self.inv_t.ctypes.data_as(C.POINTER(C.c_uint64)))

    # ---------------- transforms ----------------
    def ntt(self, a: np.ndarray, j: int) -> np.ndarray:
        """Negacyclic NTT mod q_j (products in R_q = Z_q[x]/(x^N + 1), Sec. 2.3):
        slot s = a(psi_j^(2 brv(s) + 1))."""
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        lib().oracle_ntt(a.ctypes.data_as(C.POINTER(C.c_uint64)), self.N, int(self.q[j]),
                         self.fwd[j].ctypes.data_as(C.POINTER(C.c_uint64)))
        return a

    def intt(self, a: np.ndarray, j: int) -> np.ndarray:
        """Inverse of ntt: NTT form back to coefficients mod q_j (Sec. 2.3)."""
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        lib().oracle_intt(a.ctypes.data_as(C.POINTER(C.c_uint64)), self.N, int(self.q[j]),
                          self.inv[j].ctypes.data_as(C.POINTER(C.c_uint64)))
        return a

    def ntt_t(self, a: np.ndarray) -> np.ndarray:
        """Slot values of a plaintext: the negacyclic NTT mod t."""
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        lib().oracle_ntt(a.ctypes.data_as(C.POINTER(C.c_uint64)), self.N, self.t,
                         self.fwd_t.ctypes.data_as(C.POINTER(C.c_uint64)))
        return a

    def intt_t(self, a: np.ndarray) -> np.ndarray:
        """The plaintext (coefficients in [0, t)) whose slots are a."""
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        lib().oracle_intt(a.ctypes.data_as(C.POINTER(C.c_uint64)), self.N, self.t,
                          self.inv_t.ctypes.data_as(C.POINTER(C.c_uint64)))
        return a

    def schoolbook_mod(self, a: np.ndarray, b: np.ndarray, m: int) -> np.ndarray:
        """Negacyclic product mod (x^N + 1, m) by the schoolbook loop."""
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.zeros(self.N, dtype=np.uint64)
        lib().oracle_negacyclic_schoolbook(_p(a), _p(b), self.N, int(m), _p(out))
        return out

    def schoolbook(self, a: np.ndarray, b: np.ndarray, j: int) -> np.ndarray:
        """Negacyclic product in R_q mod q_j by the schoolbook loop (the
        definition of the ring product, Sec. 5.3)."""
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.zeros(self.N, dtype=np.uint64)
        lib().oracle_negacyclic_schoolbook(_p(a), _p(b), self.N, int(self.q[j]), _p(out))
        return out

    # ---------------- protocol steps ----------------
    def keygen(self, seed: int):
        """AHE.Keygen (Pi_ls step 1): ternary s from stream (seed, 1) and its NTT
        s_hat per prime; returns (s int8 [N], s_hat [L][N])."""
        s = np.zeros(self.N, dtype=np.int8)
        s_hat = np.zeros((self.L, self.N), dtype=np.uint64)
        lib().oracle_keygen(C.byref(self._c), seed, _p(s), _p(s_hat))
        return s, s_hat

    def encrypt(self, s_hat: np.ndarray, qv: np.ndarray, seed: int, qid: int) -> np.ndarray:
        """AHE.Enc of one query (Pi_ls step 2, Sec. 5.3): coordinate i as the
        constant plaintext m_i = (t - 2 q_i) mod t, private-key BFV; returns
        ct [d][2][L][N] in NTT form."""
        qv = np.ascontiguousarray(qv, dtype=np.uint8)
        assert qv.shape == (self.d,)
        ct = np.zeros((self.d, 2, self.L, self.N), dtype=np.uint64)
        lib().oracle_encrypt(C.byref(self._c), _p(np.ascontiguousarray(s_hat)), _p(qv),
                             seed, qid, _p(ct))
        return ct

    def blocks(self, n: int) -> int:
        """Number of N-point blocks covering n points (Sec. 5.3 packs N points
        per plaintext)."""
        return (n + self.N - 1) // self.N

    def encode_db(self, coords: np.ndarray, perm: np.ndarray | None, k0: int = 0,
                  k1: int | None = None, slots: bool = False):
        """Coefficient encoding (the C loops), or slot encoding: each
        coordinate row (and the norm row) of a block becomes the plaintext
        whose CRT slots mod t it is, then its NTT per prime."""
        if slots:
            return self._encode_db_slots(coords, perm, k0, k1)
        coords = np.ascontiguousarray(coords, dtype=np.uint8)
        n = coords.shape[0] if perm is None else len(perm)
        if perm is None:
            perm = np.arange(n, dtype=np.uint32)
        perm = np.ascontiguousarray(perm, dtype=np.uint32)
        k1 = self.blocks(n) if k1 is None else k1
        nk = k1 - k0
        pt = np.zeros((nk, self.L, self.d, self.N), dtype=np.uint64)
        norms = np.zeros(nk * self.N, dtype=np.uint32)
        lib().oracle_encode_db(C.byref(self._c), _p(coords), _p(perm), n, k0, k1,
                               _p(pt), _p(norms))
        return pt, norms

    def _encode_db_slots(self, coords, perm, k0, k1):
        assert self.slots_ok
        coords = np.ascontiguousarray(coords, dtype=np.uint8)
        n = coords.shape[0] if perm is None else len(perm)
        perm = np.arange(n) if perm is None else np.asarray(perm, dtype=np.int64)
        k1 = self.blocks(n) if k1 is None else k1
        N, d = self.N, self.d
        pt = np.zeros((k1 - k0, self.L, d, N), dtype=np.uint64)
        norms = np.zeros((k1 - k0) * N, dtype=np.uint32)
        for kk, k in enumerate(range(k0, k1)):
            rows = np.zeros((N, d), dtype=np.int64)
            cnt = max(0, min(n - k * N, N))
            rows[:cnt] = coords[perm[k * N:k * N + cnt]]
            for i in range(d):
                poly = self.intt_t(rows[:, i].astype(np.uint64))
                for j in range(self.L):
                    pt[kk, j, i] = self.ntt(poly, j)
            nrm = np.sum(rows * rows, axis=1).astype(np.uint64)
            norms[kk * N:(kk + 1) * N] = self.intt_t(nrm).astype(np.uint32)
        return pt, norms

    def mask_r(self, mask_seed: int, qid: int, gpos: int) -> int:
        """The server's mask value at global position gpos: the 128-bit draw
        (stream mask_seed, purpose 4, object qid) reduced mod t."""
        lo, hi = self.draw128(mask_seed, 4, qid, gpos)
        return ((hi << 64) | lo) % self.t

    def slot_shares(self, n: int, k0: int, k1: int, mask_seed: int, qid: int) -> np.ndarray:
        """Slot encoding, the server's shares of blocks k0 .. k1: t - the
        slots of the mask polynomial R (coefficients = the mask draws of
        the block's positions, padding included)."""
        N, t = self.N, self.t
        out = []
        for k in range(k0, k1):
            R = np.array([self.mask_r(mask_seed, qid, k * N + x) for x in range(N)], dtype=np.uint64)
            Rh = self.ntt_t(R).astype(np.int64)
            cnt = max(0, min(n - k * N, N))
            out.append(((t - Rh[:cnt]) % t).astype(np.uint32))
        return np.concatenate(out) if out else np.zeros(0, dtype=np.uint32)

    def mac(self, ct: np.ndarray, pt: np.ndarray) -> np.ndarray:
        """Pi_ls step 3, sum_i CMult(c_i, g_ik) per block, slot-wise in the NTT
        domain; returns acc [nk][2][L][N]."""
        nk = pt.shape[0]
        acc = np.zeros((nk, 2, self.L, self.N), dtype=np.uint64)
        lib().oracle_mac(C.byref(self._c), _p(np.ascontiguousarray(ct)),
                         _p(np.ascontiguousarray(pt)), nk, _p(acc))
        return acc

    def intt_mask(self, acc: np.ndarray, norms: np.ndarray, n: int, k0: int, k1: int,
                  mask_seed: int, qid: int):
        """Pi_ls step 3, "+ r": each block back to coefficient form plus
        Delta (||p||^2 + r) on c0; returns (responses, server shares t - r)."""
        out = np.zeros_like(acc)
        cnt = max(0, min(n, k1 * self.N) - k0 * self.N)
        share = np.zeros(cnt, dtype=np.uint32)
        lib().oracle_intt_mask(C.byref(self._c), _p(np.ascontiguousarray(acc)),
                               _p(np.ascontiguousarray(norms, dtype=np.uint32)),
                               n, k0, k1, mask_seed, qid, _p(out), _p(share))
        return out, share

    def distances(self, ct: np.ndarray, coords: np.ndarray, perm, mask_seed: int, qid: int,
                  k0: int = 0, k1: int | None = None, pk: np.ndarray | None = None,
                  flood_bits: int = 0, slots: bool = False):
        """Pi_ls step 3 for blocks [k0, k1): encode, MAC, INTT, mask; with a
        public key also the circuit-privacy terms (re-randomisation before the
        INTT, flooding after it).  With slot encoding the server's shares are
        those of the mask polynomial's slots."""
        n = coords.shape[0] if perm is None else len(perm)
        k1 = self.blocks(n) if k1 is None else k1
        pt, norms = self.encode_db(coords, perm, k0, k1, slots=slots)
        acc = self.mac(ct, pt)
        if pk is not None:
            self.rerandomize(acc, pk, mask_seed, qid, k0)
        out, share = self.intt_mask(acc, norms, n, k0, k1, mask_seed, qid)
        if pk is not None:
            self.flood(out, mask_seed, qid, k0, flood_bits)
        if slots:
            share = self.slot_shares(n, k0, k1, mask_seed, qid)
        return out, share

    # ---------------- response form ----------------
    def to_ntt_form(self, ct_out: np.ndarray) -> np.ndarray:
        """The NTT-form response: every polynomial [k][c][j] transformed."""
        out = np.empty_like(ct_out)
        for k in range(ct_out.shape[0]):
            for c in range(2):
                for j in range(self.L):
                    out[k, c, j] = self.ntt(ct_out[k, c, j], j)
        return out

    def from_ntt_form(self, ct_ntt: np.ndarray) -> np.ndarray:
        """Inverse of to_ntt_form: every polynomial back to coefficient form."""
        out = np.empty_like(ct_ntt)
        for k in range(ct_ntt.shape[0]):
            for c in range(2):
                for j in range(self.L):
                    out[k, c, j] = self.intt(ct_ntt[k, c, j], j)
        return out

    # ---------------- circuit privacy ----------------
    def public_key(self, s_hat: np.ndarray, seed: int) -> np.ndarray:
        """The client's public key for circuit privacy (Sec. 2.3): pk1 = a,
        pk0 = -a s + e, layout [2][L][N], NTT form."""
        pk = np.zeros((2, self.L, self.N), dtype=np.uint64)
        lib().oracle_public_key(C.byref(self._c), _p(np.ascontiguousarray(s_hat)), seed, _p(pk))
        return pk

    def rerandomize(self, acc: np.ndarray, pk: np.ndarray, seed: int, qid: int, k0: int):
        """In place: acc[k] (NTT form) += pk * NTT(u) for blocks k0, k0 + 1, .."""
        assert acc.flags["C_CONTIGUOUS"]
        lib().oracle_rerandomize(C.byref(self._c), _p(acc), _p(np.ascontiguousarray(pk)), seed,
                                 qid, k0, acc.shape[0])

    def flood(self, out: np.ndarray, seed: int, qid: int, k0: int, flood_bits: int):
        """In place: c0 += e1 (uniform in [-2^F, 2^F)), c1 += e2 (CBD 21)."""
        assert out.flags["C_CONTIGUOUS"] and 0 <= flood_bits <= 255
        lib().oracle_flood(C.byref(self._c), _p(out), seed, qid, k0, out.shape[0], flood_bits)

    def max_flood_bits(self) -> int:
        """Largest F with 2^F + (structured noise) < Delta / 2 for every
        decryptable response: F <= floor(log2 Delta) - 2."""
        return self.P.delta.bit_length() - 3

    def phase_noise(self, ct_out: np.ndarray, s: np.ndarray, m: np.ndarray) -> list:
        """Exact |c0 + c1 s - Delta m| (centred mod Q) of every coefficient."""
        P = self.P
        Q = P.Q
        v = self.decrypt_phase(ct_out, s)
        coef = [(Q // qj) * pow(Q // qj, -1, qj) % Q for qj in P.q]
        out = []
        for k in range(v.shape[0]):
            cols = [v[k, j].tolist() for j in range(self.L)]
            for x in range(self.N):
                w = sum(int(cols[j][x]) * coef[j] for j in range(self.L)) % Q
                e = (w - P.delta * int(m[k * self.N + x])) % Q
                out.append(min(e, Q - e))
        return out

    def decrypt_phase(self, ct_out: np.ndarray, s: np.ndarray) -> np.ndarray:
        """First half of AHE.Dec (Pi_ls step 4): c0 + c1 s mod q_j, coefficient
        form, [nk][L][N]."""
        nk = ct_out.shape[0]
        v = np.zeros((nk, self.L, self.N), dtype=np.uint64)
        lib().oracle_decrypt_phase(C.byref(self._c), _p(np.ascontiguousarray(ct_out)),
                                   _p(np.ascontiguousarray(s, dtype=np.int8)), nk, _p(v))
        return v

    def scale_round(self, v: np.ndarray) -> np.ndarray:
        """BFV decryption's last step with exact integers: CRT the residues to
        w in [0, Q), then m = floor((t w + floor(Q/2)) / Q) mod t."""
        P = self.P
        Q, t = P.Q, P.t
        coef = []
        for qj in P.q:
            Qj = Q // qj
            coef.append(Qj * pow(Qj, -1, qj) % Q)
        flat = v.reshape(-1, self.L, self.N) if v.ndim == 3 else v
        nk = flat.shape[0]
        out = np.zeros(nk * self.N, dtype=np.int64)
        half = Q // 2
        for k in range(nk):
            cols = [flat[k, j].tolist() for j in range(self.L)]
            for x in range(self.N):
                w = sum(int(cols[j][x]) * coef[j] for j in range(self.L)) % Q
                out[k * self.N + x] = ((t * w + half) // Q) % t
        return out

    def noise_ok(self, v: np.ndarray, m: np.ndarray) -> bool:
        """Check |w - Delta m| < Delta / 4 for every coefficient (decryption
        margin): the rounding above is then unambiguous."""
        P = self.P
        Q = P.Q
        coef = [(Q // qj) * pow(Q // qj, -1, qj) % Q for qj in P.q]
        nk = v.shape[0]
        lim = P.delta // 4
        for k in range(nk):
            cols = [v[k, j].tolist() for j in range(self.L)]
            for x in range(self.N):
                w = sum(int(cols[j][x]) * coef[j] for j in range(self.L)) % Q
                e = (w - P.delta * int(m[k * self.N + x])) % Q
                if min(e, Q - e) >= lim:
                    return False
        return True

    def decrypt_shares(self, ct_out: np.ndarray, s: np.ndarray, qv: np.ndarray, n: int,
                       slots: bool = False):
        """Pi_ls step 4 plus the client's local term: sigma_C = m + ||q||^2 mod t
        for the first n positions (with slot encoding, m's slots)."""
        v = self.decrypt_phase(ct_out, s)
        m = self.scale_round(v)
        if slots:
            m = np.concatenate([self.ntt_t(m[k * self.N:(k + 1) * self.N].astype(np.uint64))
                                for k in range(len(m) // self.N)]).astype(np.int64)
        m = m[:n]
        qn = int(np.sum(np.asarray(qv, dtype=np.int64) ** 2))
        return ((m + qn) % self.t).astype(np.uint32)

    def mod_switch(self, ct_out: np.ndarray) -> np.ndarray:
        """Modulus switching of coefficient-form responses from Q = q_0 ...
        q_{L-1} down to q_0 (the standard BFV rescaling of [FV12]; not a step
        of Pi_ls, which sends the responses at the full modulus): every
        coefficient, as the integer c in [0, Q) that its residues represent,
        becomes round(q_0 c / Q) mod q_0.  [nk][2][L][N] -> [nk][2][N]."""
        P = self.P
        Q, q0 = P.Q, P.q[0]
        coef = [(Q // qj) * pow(Q // qj, -1, qj) % Q for qj in P.q]
        nk = ct_out.shape[0]
        out = np.zeros((nk, 2, self.N), dtype=np.uint64)
        for k in range(nk):
            for c in range(2):
                cols = [ct_out[k, c, j].tolist() for j in range(self.L)]
                row = []
                for x in range(self.N):
                    w = sum(int(cols[j][x]) * coef[j] for j in range(self.L)) % Q
                    row.append(((2 * q0 * w + Q) // (2 * Q)) % q0)   # round half up
                out[k, c] = row
        return out

    def prime0(self) -> "Oracle":
        """The same parameters with the first prime alone: the scheme that
        decrypts modulus-switched responses (same q_0, N and t)."""
        O1 = Oracle(self.N, 1, self.P.prime_bits, self.P.t_rule, self.d, self.b_c)
        assert O1.P.q[0] == self.P.q[0] and O1.t == self.t
        return O1

    def decrypt_shares_switched(self, ct1: np.ndarray, s: np.ndarray, qv: np.ndarray, n: int,
                                slots: bool = False):
        """Pi_ls step 4 on responses switched to q_0 ([nk][2][N]): the client's
        shares by decryption modulo q_0."""
        nk = ct1.shape[0]
        return self.prime0().decrypt_shares(ct1.reshape(nk, 2, 1, self.N), s, qv, n, slots)

    def draw128(self, seed: int, purpose: int, obj: int, c: int):
        """The 128-bit draw of coefficient c of ChaCha20 stream (seed, purpose,
        object): the randomness of every protocol step (Sec. 2.3, 5.3)."""
        out = np.zeros(2, dtype=np.uint64)
        lib().oracle_draw128(seed, purpose, obj, c, _p(out))
        return int(out[0]), int(out[1])


def chacha20_block(key_words, counter: int, nonce_words):
    """The ChaCha20 block function (RFC 8439, its section 2.3), as 16 words."""
    key = np.array(key_words, dtype=np.uint32)
    nonce = np.array(nonce_words, dtype=np.uint32)
    out = np.zeros(16, dtype=np.uint32)
    lib().oracle_chacha20_block(_p(key), counter, _p(nonce), _p(out))
    return out
