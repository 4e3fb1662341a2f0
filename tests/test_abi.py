"""CPU-only checks of the C ABI: the library builds, loads, exports every
symbol include/*.h declares, and rejects invalid parameters on the host
before touching a device."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

from paper_1904_02033_b300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(sanns_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    path = pbuild.build()
    return C.CDLL(path)


def test_header_declares_the_five_protocol_calls():
    names = declared_symbols()
    for n in ("sanns_keygen", "sanns_encode_db", "sanns_encrypt_query", "sanns_distances",
              "sanns_decrypt_shares"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only", pbuild.LIB]).decode()
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = declared_symbols() - exported
    assert not missing, missing
    for n in declared_symbols():
        getattr(lib, n)


class Params(C.Structure):
    _fields_ = [("N", C.c_uint32), ("L", C.c_uint32), ("prime_bits", C.c_uint32),
                ("t_rule", C.c_uint32), ("d", C.c_uint32), ("b_c", C.c_uint32)]


@pytest.mark.parametrize("N,L,bits,rule,d", [
    (100, 2, 54, 0, 8),      # N not a power of two
    (32768, 2, 54, 0, 8),    # N too large
    (4096, 0, 54, 0, 8),     # no primes
    (4096, 5, 54, 0, 8),     # too many primes
    (4096, 2, 61, 0, 8),     # primes too large for the lazy NTT bounds
    (4096, 2, 54, 2, 8),     # unknown t rule
    (4096, 2, 54, 0, 0),     # d = 0
    (4096, 2, 54, 0, 225),   # d above the shared-memory tile
    (4096, 1, 24, 0, 8),     # t = 16.8M does not fit below a 24-bit prime
])
def test_invalid_params_rejected_on_host(lib, N, L, bits, rule, d):
    lib.sanns_ctx_create.argtypes = [C.POINTER(Params), C.POINTER(C.c_void_p)]
    lib.sanns_last_error.restype = C.c_char_p
    h = C.c_void_p(1234)
    rc = lib.sanns_ctx_create(C.byref(Params(N, L, bits, rule, d, 8)), C.byref(h))
    assert rc == -1, lib.sanns_last_error()
    assert h.value is None
    assert lib.sanns_last_error()


def test_null_handles_rejected(lib):
    lib.sanns_distances.argtypes = [C.c_void_p] * 4 + [C.c_uint64] + [C.c_void_p] * 4
    assert lib.sanns_distances(None, None, None, 1, 0, None, None, None, None) == -1
    lib.sanns_keygen.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]
    assert lib.sanns_keygen(None, 0, None, None) == -1


def test_null_handles_rejected_by_the_seeded_and_prepared_calls(lib):
    # validated on the host before any device work, so no GPU is needed
    lib.sanns_expand_query.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint64, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
    assert lib.sanns_expand_query(None, None, 1, 0, None, None, None) == -1
    lib.sanns_gather_prepare.argtypes = [C.c_void_p] * 3 + [C.c_uint32, C.c_uint32, C.c_void_p]
    assert lib.sanns_gather_prepare(None, None, None, 1, 1, None) == -1      # out is NULL
    out = C.c_void_p(1)
    assert lib.sanns_gather_prepare(None, None, None, 1, 1, C.byref(out)) == -1
    assert out.value is None                                                # cleared on failure
    lib.sanns_distances_gather_prepared.argtypes = [C.c_void_p] * 3 + [C.c_uint64] + [C.c_void_p] * 5
    assert lib.sanns_distances_gather_prepared(None, None, None, 0, None, None, None, None, None) == -1
    lib.sanns_gather_batch_free.argtypes = [C.c_void_p]
    lib.sanns_gather_batch_free(None)                                       # a no-op
