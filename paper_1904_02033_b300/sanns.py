"""Python binding of libsanns.so (include/sanns.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Buffers are torch
tensors on the current CUDA device (uint8 / uint32 / uint64); the stream is
torch's current stream unless one is passed.  There is no fallback: if the
shared library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

_LIB = None


class SannsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sanns error {code}: {msg}")
        self.code = code


class _Params(C.Structure):
    _fields_ = [("N", C.c_uint32), ("L", C.c_uint32), ("prime_bits", C.c_uint32),
                ("t_rule", C.c_uint32), ("d", C.c_uint32), ("b_c", C.c_uint32)]


_VP = C.c_void_p
_SIGS = {
    "sanns_last_error": ([], C.c_char_p),
    "sanns_device_sms": ([], C.c_int),
    "sanns_ctx_create": ([C.POINTER(_Params), C.POINTER(_VP)], C.c_int),
    "sanns_ctx_free": ([_VP], None),
    "sanns_ctx_query": ([_VP, _VP, _VP, _VP, _VP], C.c_int),
    "sanns_ntt": ([_VP, _VP, C.c_uint64, C.c_int, _VP], C.c_int),
    "sanns_keygen": ([_VP, C.c_uint64, C.POINTER(_VP), _VP], C.c_int),
    "sanns_sk_free": ([_VP], None),
    "sanns_sk_export": ([_VP, _VP, _VP, _VP], C.c_int),
    "sanns_encode_db": ([_VP, _VP, C.c_uint64, _VP, C.c_uint64, C.POINTER(_VP), _VP], C.c_int),
    "sanns_db_free": ([_VP], None),
    "sanns_db_info": ([_VP, _VP, _VP], C.c_int),
    "sanns_db_set_position_base": ([_VP, C.c_uint64], C.c_int),
    "sanns_db_export": ([_VP, C.c_uint64, C.c_uint64, _VP, _VP, _VP], C.c_int),
    "sanns_db_import": ([_VP, C.c_uint64, _VP, _VP, C.POINTER(_VP), _VP], C.c_int),
    "sanns_encrypt_query": ([_VP, _VP, _VP, C.c_uint32, C.c_uint64, _VP, _VP, _VP], C.c_int),
    "sanns_expand_query": ([_VP, _VP, C.c_uint32, C.c_uint64, _VP, _VP, _VP], C.c_int),
    "sanns_distances": ([_VP, _VP, _VP, C.c_uint32, C.c_uint64, _VP, _VP, _VP, _VP], C.c_int),
    "sanns_distances_mac": ([_VP, _VP, _VP, C.c_uint32, _VP, _VP], C.c_int),
    "sanns_distances_finish": ([_VP, _VP, C.c_uint32, C.c_uint64, _VP, _VP, _VP, _VP], C.c_int),
    "sanns_clusters_create": ([_VP, _VP, C.c_uint64, _VP, _VP, C.c_uint32, C.POINTER(_VP), _VP],
                              C.c_int),
    "sanns_clusters_free": ([_VP], None),
    "sanns_gather_plan": ([_VP, _VP, C.c_uint32, C.c_uint32, _VP, _VP], C.c_int),
    "sanns_distances_gather": ([_VP, _VP, _VP, C.c_uint32, _VP, C.c_uint32, C.c_uint64, _VP, _VP,
                                _VP, _VP, _VP], C.c_int),
    "sanns_gather_prepare": ([_VP, _VP, _VP, C.c_uint32, C.c_uint32, C.POINTER(_VP)], C.c_int),
    "sanns_gather_batch_free": ([_VP], None),
    "sanns_distances_gather_prepared": ([_VP, _VP, _VP, C.c_uint64, _VP, _VP, _VP, _VP, _VP], C.c_int),
    "sanns_decrypt_shares_noalloc": ([_VP, _VP, _VP, C.c_uint32, C.c_uint64, _VP, _VP, _VP],
                                     C.c_int),
    "sanns_decrypt_noalloc_max_words": ([], C.c_uint64),
    "sanns_mac_variants": ([], C.c_int),
    "sanns_mac_variant_name": ([C.c_int], C.c_char_p),
    "sanns_set_mac_variant": ([_VP, C.c_int], C.c_int),
    "sanns_set_mac_sms": ([_VP, C.c_int], C.c_int),
    "sanns_autotune_mac": ([_VP, _VP, _VP, C.c_uint32, _VP, C.c_int, _VP, _VP], C.c_int),
    "sanns_autotune_batched": ([_VP, _VP, _VP, C.c_uint32, _VP, C.c_int, _VP, _VP], C.c_int),
    "sanns_public_key": ([_VP, _VP, C.c_uint64, _VP, _VP], C.c_int),
    "sanns_set_encoding": ([_VP, C.c_int], C.c_int),
    "sanns_selftest_wait_timeout": ([_VP, C.c_uint32, _VP], C.c_int),
    "sanns_set_response_form": ([_VP, C.c_int], C.c_int),
    "sanns_set_response_primes": ([_VP, C.c_uint32], C.c_int),
    "sanns_copy_responses": ([_VP, _VP, C.c_uint32, C.c_uint64, _VP, _VP], C.c_int),
    "sanns_topk": ([_VP, _VP, _VP, C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32, _VP,
                    _VP, _VP], C.c_int),
    "sanns_topk_segments": ([_VP, _VP, _VP, C.c_uint32, _VP, _VP, _VP, _VP, _VP, C.c_uint32,
                             C.c_uint64, C.c_uint32, _VP, _VP, _VP], C.c_int),
    "sanns_circuit_privacy_max_flood_bits": ([_VP], C.c_int),
    "sanns_set_circuit_privacy": ([_VP, _VP, C.c_uint32, _VP], C.c_int),
    "sanns_db_prepare_batched": ([_VP, _VP, _VP], C.c_int),
    "sanns_distances_batched": ([_VP, _VP, _VP, C.c_uint32, C.c_uint64, _VP, _VP, _VP, _VP],
                                C.c_int),
    "sanns_distances_batched_mac": ([_VP, _VP, _VP, C.c_uint32, _VP, _VP], C.c_int),
    "sanns_device_status": ([_VP, _VP], C.c_int),
    "sanns_measure_mma_rates": ([_VP, _VP, _VP], C.c_int),
    "sanns_distances_scratch_bytes": ([_VP, C.c_uint32, C.c_int, C.POINTER(C.c_uint64)], C.c_int),
    "sanns_measure_int_rates": ([_VP, _VP, _VP], C.c_int),
    "sanns_batched_tune": ([_VP, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                            C.c_uint32, C.c_uint32], C.c_int),
    "sanns_decrypt_shares": ([_VP, _VP, _VP, C.c_uint32, C.c_uint64, _VP, _VP, _VP], C.c_int),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libsanns.so (built by __graft_entry__.build() / build.py)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: build it with paper_1904_02033_b300.build")
        _build.build()
    lib = C.CDLL(path)
    for name, (args, res) in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _LIB = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise SannsError(rc, load().sanns_last_error().decode())


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Context:
    def __init__(self, handle, N, L, prime_bits, t_rule, d, b_c):
        self.handle = handle
        self.N, self.L, self.prime_bits, self.t_rule, self.d, self.b_c = (
            N, L, prime_bits, t_rule, d, b_c)
        self.response_primes = L

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.sanns_ctx_free(self.handle)
            self.handle = None

    def query(self) -> dict:
        q = (C.c_uint64 * self.L)()
        psi = (C.c_uint64 * self.L)()
        dl = (C.c_uint64 * self.L)()
        t = C.c_uint64()
        _check(load().sanns_ctx_query(self.handle, q, psi, C.byref(t), dl))
        return {"q": list(q), "psi": list(psi), "t": t.value, "delta": list(dl)}


class SecretKey:
    def __init__(self, handle, ctx):
        self.handle, self.ctx = handle, ctx

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.sanns_sk_free(self.handle)
            self.handle = None


class Database:
    def __init__(self, handle, ctx, n, K):
        self.handle, self.ctx, self.n, self.K = handle, ctx, n, K

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.sanns_db_free(self.handle)
            self.handle = None


class Clusters:
    def __init__(self, handle, ctx, n, C, offsets):
        self.handle, self.ctx, self.n, self.C, self.offsets = handle, ctx, n, C, offsets

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.sanns_clusters_free(self.handle)
            self.handle = None


def sanns_device_sms() -> int:
    return load().sanns_device_sms()


def sanns_ctx_create(N: int, L: int, prime_bits: int, t_rule: int, d: int, b_c: int = 8) -> Context:
    p = _Params(N, L, prime_bits, t_rule, d, b_c)
    h = _VP()
    _check(load().sanns_ctx_create(C.byref(p), C.byref(h)))
    return Context(h, N, L, prime_bits, t_rule, d, b_c)


def sanns_ntt(ctx: Context, data: torch.Tensor, inverse: bool = False, stream=None):
    assert data.dtype == torch.uint64 and data.numel() % (ctx.L * ctx.N) == 0
    count = data.numel() // (ctx.L * ctx.N)
    _check(load().sanns_ntt(ctx.handle, _ptr(data), count, 1 if inverse else 0, _stream(stream)))
    return data


def sanns_keygen(ctx: Context, seed: int, stream=None) -> SecretKey:
    h = _VP()
    _check(load().sanns_keygen(ctx.handle, seed, C.byref(h), _stream(stream)))
    return SecretKey(h, ctx)


def sanns_sk_export(sk: SecretKey, stream=None):
    ctx = sk.ctx
    s = torch.empty(ctx.N, dtype=torch.int8, device="cuda")
    s_hat = torch.empty((ctx.L, ctx.N), dtype=torch.uint64, device="cuda")
    _check(load().sanns_sk_export(sk.handle, _ptr(s), _ptr(s_hat), _stream(stream)))
    return s, s_hat


def sanns_encode_db(ctx: Context, coords: torch.Tensor, perm: torch.Tensor | None = None,
                    n: int | None = None, stream=None) -> Database:
    assert coords.dtype == torch.uint8 and coords.dim() == 2 and coords.shape[1] == ctx.d
    if perm is not None:
        assert perm.dtype == torch.uint32
        n = perm.numel() if n is None else n
    else:
        n = coords.shape[0] if n is None else n
    h = _VP()
    _check(load().sanns_encode_db(ctx.handle, _ptr(coords), coords.shape[0], _ptr(perm), n,
                                  C.byref(h), _stream(stream)))
    K = (n + ctx.N - 1) // ctx.N
    return Database(h, ctx, n, K)


def sanns_db_export(db: Database, k0: int = 0, k1: int | None = None, stream=None):
    ctx = db.ctx
    k1 = db.K if k1 is None else k1
    pt = torch.empty((k1 - k0, ctx.L, ctx.d, ctx.N), dtype=torch.uint64, device="cuda")
    norms = torch.empty((k1 - k0) * ctx.N, dtype=torch.uint32, device="cuda")
    _check(load().sanns_db_export(db.handle, k0, k1, _ptr(pt), _ptr(norms), _stream(stream)))
    return pt, norms


def sanns_db_import(ctx: Context, n: int, pt: torch.Tensor, norms: torch.Tensor,
                    stream=None) -> Database:
    """A database from exported plaintexts [K][L][d][N] (canonical residues,
    NTT form) and norms [K N] (CUDA tensors), K = ceil(n / N)."""
    K = (n + ctx.N - 1) // ctx.N
    assert pt.dtype == torch.uint64 and tuple(pt.shape) == (K, ctx.L, ctx.d, ctx.N)
    assert norms.dtype == torch.uint32 and norms.numel() == K * ctx.N
    h = _VP()
    _check(load().sanns_db_import(ctx.handle, n, _ptr(pt), _ptr(norms), C.byref(h), _stream(stream)))
    return Database(h, ctx, n, K)


def sanns_encrypt_query(ctx: Context, sk: SecretKey, q: torch.Tensor, seed: int,
                        qids: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    assert q.dtype == torch.uint8 and q.dim() == 2 and q.shape[1] == ctx.d
    B = q.shape[0]
    assert qids.dtype == torch.uint64 and qids.numel() == B
    if out is None:
        out = torch.empty((B, ctx.d, 2, ctx.L, ctx.N), dtype=torch.uint64, device="cuda")
    _check(load().sanns_encrypt_query(ctx.handle, sk.handle, _ptr(q), B, seed, _ptr(qids),
                                      _ptr(out), _stream(stream)))
    return out


def sanns_expand_query(ctx: Context, c0: torch.Tensor, seed: int, qids: torch.Tensor,
                       out: torch.Tensor | None = None, stream=None):
    """Rebuild query ciphertexts [B][d][2][L][N] from their c0 components
    [B][d][L][N] and the encryption seed (c1 is the seed's stream)."""
    assert c0.dtype == torch.uint64 and c0.is_contiguous()
    B = c0.shape[0]
    assert c0.shape == (B, ctx.d, ctx.L, ctx.N)
    assert qids.dtype == torch.uint64 and qids.numel() == B
    if out is None:
        out = torch.empty((B, ctx.d, 2, ctx.L, ctx.N), dtype=torch.uint64, device="cuda")
    _check(load().sanns_expand_query(ctx.handle, _ptr(c0), B, seed, _ptr(qids), _ptr(out),
                                     _stream(stream)))
    return out


def sanns_distances(ctx: Context, db: Database, ct_in: torch.Tensor, mask_seed: int,
                    qids: torch.Tensor, ct_out: torch.Tensor | None = None,
                    srv_share: torch.Tensor | None = None, stream=None):
    assert ct_in.dtype == torch.uint64
    B = ct_in.shape[0]
    assert ct_in.shape == (B, ctx.d, 2, ctx.L, ctx.N)
    assert qids.dtype == torch.uint64 and qids.numel() == B
    if ct_out is None:
        ct_out = torch.empty((B, db.K, 2, ctx.L, ctx.N), dtype=torch.uint64, device="cuda")
    if srv_share is None:
        srv_share = torch.empty((B, db.n), dtype=torch.uint32, device="cuda")
    _check(load().sanns_distances(ctx.handle, db.handle, _ptr(ct_in), B, mask_seed, _ptr(qids),
                                  _ptr(ct_out), _ptr(srv_share), _stream(stream)))
    return ct_out, srv_share


def sanns_distances_mac(ctx: Context, db: Database, ct_in: torch.Tensor,
                        ct_out: torch.Tensor | None = None, stream=None):
    B = ct_in.shape[0]
    assert ct_in.dtype == torch.uint64 and ct_in.shape == (B, ctx.d, 2, ctx.L, ctx.N)
    if ct_out is None:
        ct_out = torch.empty((B, db.K, 2, ctx.L, ctx.N), dtype=torch.uint64, device="cuda")
    _check(load().sanns_distances_mac(ctx.handle, db.handle, _ptr(ct_in), B, _ptr(ct_out),
                                      _stream(stream)))
    return ct_out


def sanns_distances_finish(ctx: Context, db: Database, ct_out: torch.Tensor, mask_seed: int,
                           qids: torch.Tensor, srv_share: torch.Tensor | None = None,
                           stream=None):
    B = ct_out.shape[0]
    assert ct_out.dtype == torch.uint64 and ct_out.shape == (B, db.K, 2, ctx.L, ctx.N)
    assert qids.dtype == torch.uint64 and qids.numel() == B
    if srv_share is None:
        srv_share = torch.empty((B, db.n), dtype=torch.uint32, device="cuda")
    _check(load().sanns_distances_finish(ctx.handle, db.handle, B, mask_seed, _ptr(qids),
                                         _ptr(ct_out), _ptr(srv_share), _stream(stream)))
    return ct_out, srv_share


def sanns_decrypt_shares(ctx: Context, sk: SecretKey, ct_out: torch.Tensor, n: int,
                         q: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    B = ct_out.shape[0]
    assert q.dtype == torch.uint8 and q.shape == (B, ctx.d)
    if out is None:
        out = torch.empty((B, n), dtype=torch.uint32, device="cuda")
    _check(load().sanns_decrypt_shares(ctx.handle, sk.handle, _ptr(ct_out), B, n, _ptr(q),
                                       _ptr(out), _stream(stream)))
    return out


def sanns_clusters_create(ctx: Context, coords: torch.Tensor, offsets, members: torch.Tensor,
                          stream=None) -> Clusters:
    """coords uint8 [n][d] (CUDA), offsets uint64 [C+1] (numpy, host), members
    uint32 (CUDA)."""
    import numpy as np
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    assert coords.dtype == torch.uint8 and coords.shape[1] == ctx.d
    assert members.dtype == torch.uint32
    h = _VP()
    _check(load().sanns_clusters_create(ctx.handle, _ptr(coords), coords.shape[0],
                                        off.ctypes.data_as(C.c_void_p), _ptr(members),
                                        len(off) - 1, C.byref(h), _stream(stream)))
    return Clusters(h, ctx, coords.shape[0], len(off) - 1, off)


def sanns_gather_plan(cl: Clusters, probes):
    """probes: numpy uint32 [B][P] -> (n_b, blocks_b) numpy uint64 arrays."""
    import numpy as np
    pr = np.ascontiguousarray(probes, dtype=np.uint32)
    B, P = pr.shape
    n_b = np.zeros(B, dtype=np.uint64)
    k_b = np.zeros(B, dtype=np.uint64)
    _check(load().sanns_gather_plan(cl.handle, pr.ctypes.data_as(C.c_void_p), B, P,
                                    n_b.ctypes.data_as(C.c_void_p),
                                    k_b.ctypes.data_as(C.c_void_p)))
    return n_b, k_b


def sanns_distances_gather(ctx: Context, cl: Clusters, ct_in: torch.Tensor, probes,
                           mask_seed: int, qids: torch.Tensor, with_ids: bool = True,
                           stream=None):
    """Returns (ct_out [sum K_b][2][L][N], srv_share [sum n_b], ids [sum n_b] or
    None, n_b, blocks_b)."""
    import numpy as np
    pr = np.ascontiguousarray(probes, dtype=np.uint32)
    B, P = pr.shape
    assert ct_in.dtype == torch.uint64 and ct_in.shape == (B, ctx.d, 2, ctx.L, ctx.N)
    n_b, k_b = sanns_gather_plan(cl, pr)
    tot_k, tot_n = int(k_b.sum()), int(n_b.sum())
    ct_out = torch.empty((max(tot_k, 1), 2, ctx.L, ctx.N), dtype=torch.uint64, device="cuda")
    srv = torch.empty(max(tot_n, 1), dtype=torch.uint32, device="cuda")
    ids = torch.empty(max(tot_n, 1), dtype=torch.uint32, device="cuda") if with_ids else None
    _check(load().sanns_distances_gather(ctx.handle, cl.handle, _ptr(ct_in), B,
                                         pr.ctypes.data_as(C.c_void_p), P, mask_seed, _ptr(qids),
                                         _ptr(ct_out), _ptr(srv), _ptr(ids), _stream(stream)))
    return ct_out[:tot_k], srv[:tot_n], (ids[:tot_n] if with_ids else None), n_b, k_b


class GatherBatch:
    def __init__(self, handle, ctx, cl, n_b, k_b):
        self.handle, self.ctx, self.cl, self.n_b, self.k_b = handle, ctx, cl, n_b, k_b

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.sanns_gather_batch_free(self.handle)
            self.handle = None


def sanns_gather_prepare(ctx: Context, cl: Clusters, probes) -> GatherBatch:
    """Plan and upload one batch of probes (B x P, host) once."""
    import numpy as np
    pr = np.ascontiguousarray(probes, dtype=np.uint32)
    B, P = pr.shape
    n_b, k_b = sanns_gather_plan(cl, pr)
    h = _VP()
    _check(load().sanns_gather_prepare(ctx.handle, cl.handle, pr.ctypes.data_as(C.c_void_p), B, P,
                                       C.byref(h)))
    return GatherBatch(h, ctx, cl, n_b, k_b)


def sanns_distances_gather_prepared(ctx: Context, batch: GatherBatch, ct_in: torch.Tensor,
                                    mask_seed: int, qids: torch.Tensor, ct_out: torch.Tensor,
                                    srv_share: torch.Tensor, ids: torch.Tensor | None = None,
                                    stream=None):
    """sanns_distances_gather over a prepared batch, into caller-allocated
    outputs sized by the batch (kernels and stream-ordered scratch only, so
    the call can be captured into a CUDA graph)."""
    B = len(batch.n_b)
    assert ct_in.dtype == torch.uint64 and ct_in.shape == (B, ctx.d, 2, ctx.L, ctx.N)
    assert qids.dtype == torch.uint64 and qids.numel() == B
    assert ct_out.shape[0] >= int(batch.k_b.sum()) and srv_share.numel() >= int(batch.n_b.sum())
    _check(load().sanns_distances_gather_prepared(ctx.handle, batch.handle, _ptr(ct_in), mask_seed,
                                                  _ptr(qids), _ptr(ct_out), _ptr(srv_share), _ptr(ids),
                                                  _stream(stream)))
    return ct_out, srv_share, ids


def sanns_decrypt_shares_noalloc(ctx: Context, sk: SecretKey, ct_out: torch.Tensor, n: int,
                                 q: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Decryption that allocates no device memory inside the call (its scratch
    is a fixed 32 MiB device array); `out` must be preallocated by callers
    that cannot allocate at all."""
    B = ct_out.shape[0]
    assert q.dtype == torch.uint8 and q.shape == (B, ctx.d)
    if out is None:
        out = torch.empty((B, n), dtype=torch.uint32, device="cuda")
    _check(load().sanns_decrypt_shares_noalloc(ctx.handle, sk.handle, _ptr(ct_out), B, n,
                                               _ptr(q), _ptr(out), _stream(stream)))
    return out


def sanns_decrypt_noalloc_max_words() -> int:
    return load().sanns_decrypt_noalloc_max_words()


def sanns_mac_variants() -> list[str]:
    lib = load()
    return [lib.sanns_mac_variant_name(v).decode() for v in range(lib.sanns_mac_variants())]


def sanns_set_mac_variant(ctx: Context, variant: int):
    _check(load().sanns_set_mac_variant(ctx.handle, variant))


def sanns_set_mac_sms(ctx: Context, sms: int):
    """SMs the MAC kernel uses (0: all); the rest stay free for concurrent
    work on other streams."""
    _check(load().sanns_set_mac_sms(ctx.handle, sms))


def sanns_autotune_mac(ctx: Context, db: Database, ct_in: torch.Tensor, ct_out: torch.Tensor,
                       reps: int = 3, stream=None):
    """Times every MAC launch variant, keeps the fastest; returns (index, ms list)."""
    n = load().sanns_mac_variants()
    ms = (C.c_float * n)()
    B = ct_in.shape[0]
    rc = load().sanns_autotune_mac(ctx.handle, db.handle, _ptr(ct_in), B, _ptr(ct_out), reps, ms,
                                   _stream(stream))
    if rc < 0:
        _check(rc)
    return rc, list(ms)


def sanns_selftest_wait_timeout(ctx: Context, limit_ms: int = 20, stream=None):
    """Runs one bounded device-side wait that must time out after limit_ms;
    the next sanns_device_status then raises SannsError with SANNS_ETIMEOUT."""
    _check(load().sanns_selftest_wait_timeout(ctx.handle, limit_ms, _stream(stream)))


def sanns_set_encoding(ctx: Context, slots: bool):
    """Slot encoding (True, needs t = 1 mod 2N) or coefficient encoding
    (False, default) for databases encoded from now on and for decryption."""
    _check(load().sanns_set_encoding(ctx.handle, 1 if slots else 0))


def sanns_set_response_form(ctx: Context, ntt: bool):
    """Responses in NTT form (True) or coefficient form (False, default)."""
    _check(load().sanns_set_response_form(ctx.handle, 1 if ntt else 0))


def sanns_set_response_primes(ctx: Context, primes: int):
    """Responses switched down to q_0 (1) or kept at every prime (ctx.L,
    default)."""
    _check(load().sanns_set_response_primes(ctx.handle, primes))
    ctx.response_primes = primes


def sanns_copy_responses(ctx: Context, ct_out: torch.Tensor, dst: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """The responses a distance call left in ct_out [B][K][2][L][N], compact:
    [B][K][2][R][N] with R = ctx.response_primes, into dst (device or pinned
    host memory; a new device tensor when None)."""
    B, K = ct_out.shape[0], ct_out.shape[1]
    shape = (B, K, 2, ctx.response_primes, ctx.N)
    if dst is None:
        dst = torch.empty(shape, dtype=torch.uint64, device="cuda")
    assert tuple(dst.shape) == shape and dst.is_contiguous() and dst.dtype == torch.uint64
    if dst.is_cuda:
        dp = _ptr(dst)
    elif dst.is_pinned():
        dp = C.c_void_p(dst.data_ptr())
    else:
        raise ValueError("dst must be a CUDA tensor or pinned host memory")
    _check(load().sanns_copy_responses(ctx.handle, _ptr(ct_out), B, K, dp, _stream(stream)))
    return dst


def sanns_topk(ctx: Context, cli_share: torch.Tensor, srv_share: torch.Tensor, k: int,
               bins: int = 0, shift: int = 0, stream=None):
    """The k smallest reconstructed distances >> shift per query: exact
    (bins = 0) or ApproxTopk over `bins` bins.  Returns (dist [B][k] uint32,
    pos [B][k] int64)."""
    assert cli_share.dtype == torch.uint32 and srv_share.dtype == torch.uint32
    assert cli_share.shape == srv_share.shape and cli_share.dim() == 2
    B, n = cli_share.shape
    dist = torch.empty((B, k), dtype=torch.uint32, device="cuda")
    pos = torch.empty((B, k), dtype=torch.int64, device="cuda")
    _check(load().sanns_topk(ctx.handle, _ptr(cli_share), _ptr(srv_share), B, n, k, bins, shift,
                             _ptr(dist), _ptr(pos), _stream(stream)))
    return dist, pos


def sanns_topk_segments(ctx: Context, cli_share: torch.Tensor, srv_share: torch.Tensor, cli_off,
                        srv_off, lengths, k: int, bins: int = 0, shift: int = 0, k_seg=None,
                        bins_seg=None, stream=None):
    """Selection over ragged lists: list b is lengths[b] elements at cli_off[b]
    (client shares) and srv_off[b] (server shares), k_seg[b] winners over
    bins_seg[b] bins where given; offsets, lengths, k_seg and bins_seg are
    host sequences.  Returns (dist [B][k] uint32, pos [B][k] int64, positions
    from the list's start; entries past a list's winners hold dist 2^32 - 1,
    pos -1)."""
    import numpy as np
    ks = None if k_seg is None else np.ascontiguousarray(k_seg, dtype=np.uint32)
    bs = None if bins_seg is None else np.ascontiguousarray(bins_seg, dtype=np.uint64)
    assert cli_share.dtype == torch.uint32 and srv_share.dtype == torch.uint32
    co = np.ascontiguousarray(cli_off, dtype=np.uint64)
    so = np.ascontiguousarray(srv_off, dtype=np.uint64)
    ln = np.ascontiguousarray(lengths, dtype=np.uint64)
    B = len(ln)
    assert len(co) == B and len(so) == B
    assert (ks is None or len(ks) == B) and (bs is None or len(bs) == B)
    assert int((co + ln).max(initial=0)) <= cli_share.numel()
    assert int((so + ln).max(initial=0)) <= srv_share.numel()
    dist = torch.empty((B, k), dtype=torch.uint32, device="cuda")
    pos = torch.empty((B, k), dtype=torch.int64, device="cuda")
    _check(load().sanns_topk_segments(ctx.handle, _ptr(cli_share), _ptr(srv_share), B,
                                      co.ctypes.data_as(C.c_void_p), so.ctypes.data_as(C.c_void_p),
                                      ln.ctypes.data_as(C.c_void_p),
                                      None if ks is None else ks.ctypes.data_as(C.c_void_p),
                                      None if bs is None else bs.ctypes.data_as(C.c_void_p),
                                      k, bins, shift, _ptr(dist), _ptr(pos), _stream(stream)))
    return dist, pos


def sanns_public_key(ctx: Context, sk: SecretKey, seed: int, stream=None) -> torch.Tensor:
    """The client's public key (-a s + e, a), [2][L][N] NTT form, for circuit privacy."""
    pk = torch.empty((2, ctx.L, ctx.N), dtype=torch.uint64, device="cuda")
    _check(load().sanns_public_key(ctx.handle, sk.handle, seed, _ptr(pk), _stream(stream)))
    return pk


def sanns_circuit_privacy_max_flood_bits(ctx: Context) -> int:
    rc = load().sanns_circuit_privacy_max_flood_bits(ctx.handle)
    if rc < 0:
        _check(rc)
    return rc


def sanns_set_circuit_privacy(ctx: Context, pk: torch.Tensor | None, flood_bits: int = 0,
                              stream=None):
    """Re-randomise and flood every later response of this context (pk = None: off)."""
    if pk is not None:
        assert pk.dtype == torch.uint64 and pk.shape == (2, ctx.L, ctx.N) and pk.is_contiguous()
    _check(load().sanns_set_circuit_privacy(ctx.handle, _ptr(pk), flood_bits, _stream(stream)))


BATCHED_CONFIGS = [(tile, pf) for tile in range(9) for pf in (0, 1)]  # index = 2 tile + prefetch


def sanns_autotune_batched(ctx: Context, db: Database, ct_in: torch.Tensor, ct_out: torch.Tensor,
                           reps: int = 2, stream=None):
    """Times the batched MAC's (tile shape, L2 prefetch) configurations, keeps
    the fastest; returns (index into BATCHED_CONFIGS, ms list)."""
    ms = (C.c_float * len(BATCHED_CONFIGS))()
    B = ct_in.shape[0]
    rc = load().sanns_autotune_batched(ctx.handle, db.handle, _ptr(ct_in), B, _ptr(ct_out), reps, ms,
                                       _stream(stream))
    if rc < 0:
        _check(rc)
    return rc, list(ms)


def sanns_db_prepare_batched(ctx: Context, db: Database, stream=None):
    _check(load().sanns_db_prepare_batched(ctx.handle, db.handle, _stream(stream)))


def sanns_distances_batched(ctx: Context, db: Database, ct_in: torch.Tensor, mask_seed: int,
                            qids: torch.Tensor, ct_out: torch.Tensor | None = None,
                            srv_share: torch.Tensor | None = None, stream=None):
    B = ct_in.shape[0]
    assert ct_in.dtype == torch.uint64 and ct_in.shape == (B, ctx.d, 2, ctx.L, ctx.N)
    assert qids.dtype == torch.uint64 and qids.numel() == B
    if ct_out is None:
        ct_out = torch.empty((B, db.K, 2, ctx.L, ctx.N), dtype=torch.uint64, device="cuda")
    if srv_share is None:
        srv_share = torch.empty((B, db.n), dtype=torch.uint32, device="cuda")
    _check(load().sanns_distances_batched(ctx.handle, db.handle, _ptr(ct_in), B, mask_seed,
                                          _ptr(qids), _ptr(ct_out), _ptr(srv_share),
                                          _stream(stream)))
    return ct_out, srv_share


def sanns_distances_batched_mac(ctx: Context, db: Database, ct_in: torch.Tensor,
                                ct_out: torch.Tensor | None = None, stream=None):
    B = ct_in.shape[0]
    assert ct_in.dtype == torch.uint64 and ct_in.shape == (B, ctx.d, 2, ctx.L, ctx.N)
    if ct_out is None:
        ct_out = torch.empty((B, db.K, 2, ctx.L, ctx.N), dtype=torch.uint64, device="cuda")
    _check(load().sanns_distances_batched_mac(ctx.handle, db.handle, _ptr(ct_in), B, _ptr(ct_out),
                                              _stream(stream)))
    return ct_out


def sanns_device_status(ctx: Context, stream=None):
    _check(load().sanns_device_status(ctx.handle, _stream(stream)))


def sanns_distances_scratch_bytes(ctx: Context, B: int, batched: bool) -> int:
    """Stream-ordered scratch one distance call with B queries allocates."""
    v = C.c_uint64()
    _check(load().sanns_distances_scratch_bytes(ctx.handle, B, 1 if batched else 0, C.byref(v)))
    return v.value


def sanns_measure_int_rates(ctx: Context, stream=None) -> dict:
    """Register-resident butterflies per second (inverse and forward) on the
    context's first prime: the integer-pipe ceiling of the transforms."""
    r = (C.c_double * 2)()
    _check(load().sanns_measure_int_rates(ctx.handle, r, _stream(stream)))
    return {"inv_butterflies_per_s": r[0], "fwd_butterflies_per_s": r[1]}


def sanns_measure_mma_rates(ctx: Context, stream=None) -> dict:
    """Measured dense tensor-core rates of this GPU: tcgen05 kind::f16 and
    legacy mma.sync f16 (TFLOP/s), legacy mma.sync s8 (TOP/s)."""
    r = (C.c_double * 3)()
    _check(load().sanns_measure_mma_rates(ctx.handle, r, _stream(stream)))
    return {"tcgen05_f16_tflops": r[0], "mma_sync_f16_tflops": r[1], "mma_sync_s8_tops": r[2]}


def sanns_batched_tune(ctx: Context, tma_ns: int = 0, mma_ns: int = 0, producer_ns: int = 32,
                       epilogue_ns: int = 128, prefetch_units: int = 0, scratch_mib: int = 4096,
                       tile: int = 7):
    _check(load().sanns_batched_tune(ctx.handle, tma_ns, mma_ns, producer_ns, epilogue_ns,
                                     prefetch_units, scratch_mib, tile))


def sanns_db_set_position_base(db: Database, pos0: int):
    _check(load().sanns_db_set_position_base(db.handle, pos0))
    db.pos0 = pos0
