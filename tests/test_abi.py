"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports
every symbol the public headers declare, and its host-only helpers agree
with the oracle.  No compute call is made here (there is no GPU)."""
import ctypes
import glob
import os
import re

import pytest

import oracle
from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_2506_00528_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        text = re.sub(r"^\s*#[^\n]*", " ", text, flags=re.M)   # preprocessor lines
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(([^;{}]*)\)\s*;", text):
            name = m.group(1)
            if name not in ("if", "while", "for", "sizeof", "return"):
                names.add(name)
    return sorted(names)


def test_header_declares_the_boundary_calls():
    names = _declared_functions()
    for required in ("evp_encode", "ternary_knn", "ternary_knn_workspace", "rerank",
                     "evp_words", "evp_default_x", "evp_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2506_00528_gb300 import evp
    assert set(_declared_functions()) <= set(evp.SIGNATURES), \
        set(_declared_functions()) - set(evp.SIGNATURES)


def test_host_helpers_match_oracle(lib):
    lib.evp_default_x.restype = ctypes.c_int32
    lib.evp_words.restype = ctypes.c_int32
    for d in list(range(1, 3001)) + [4096, 8191, 100000]:
        assert lib.evp_default_x(d) == oracle.default_x(d), d
        assert lib.evp_words(d) == oracle.words(d)
    assert lib.evp_default_x(0) == 0 and lib.evp_words(0) == 0


def test_status_strings(lib):
    lib.evp_status_string.restype = ctypes.c_char_p
    for code in range(8):
        s = lib.evp_status_string(code).decode()
        assert s.startswith("EVP_")
    assert b"UNKNOWN" in lib.evp_status_string(99)


def test_argument_errors_detected_on_host(lib):
    """Invalid arguments are rejected before any CUDA call (works without a GPU)."""
    lib.evp_encode.restype = ctypes.c_int32
    P = ctypes.c_void_p
    fake = P(0x1000)
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    # x > d, x < 1, d < 1
    assert lib.evp_encode(fake, i64(4), i32(8), i32(9), fake, None, None) == 1
    assert lib.evp_encode(fake, i64(4), i32(8), i32(0), fake, None, None) == 1
    assert lib.evp_encode(fake, i64(4), i32(0), i32(1), fake, None, None) == 1
    # d above the encode limit
    assert lib.evp_encode(fake, i64(4), i32(4096), i32(5), fake, None, None) == 6
    # n == 0 is a no-op
    assert lib.evp_encode(None, i64(0), i32(8), i32(3), None, None, None) == 0
    lib.ternary_knn.restype = ctypes.c_int32
    sz = ctypes.c_size_t
    # k > ns
    assert lib.ternary_knn(fake, i64(1), fake, i64(5), i32(8), i32(3), i32(6), fake, fake,
                           fake, sz(1 << 20), None, None) == 1
    # d above the scan limit
    assert lib.ternary_knn(fake, i64(1), fake, i64(5), i32(2000), i32(3), i32(2), fake, fake,
                           fake, sz(1 << 20), None, None) == 6
    # misaligned database pointer
    assert lib.ternary_knn(fake, i64(1), P(0x1008), i64(5), i32(8), i32(3), i32(2), fake, fake,
                           fake, sz(1 << 20), None, None) == 1
    lib.rerank.restype = ctypes.c_int32
    # k > n
    assert lib.rerank(fake, i64(1), fake, i64(5), i32(8), fake, i32(3), i32(4), fake, fake,
                      None, None) == 1


@pytest.mark.parametrize("d,ns", [(384, 20_000), (768, 10_000_000), (1024, 3_000)])
def test_workspace_serves_every_smaller_batch(lib, d, ns):
    """The workspace size returned for nq queries is enough for any call with
    fewer queries (servers and batch plans size one buffer for the largest
    batch): it never decreases as nq grows, on every path and for every k."""
    f = lib.ternary_knn_path_workspace
    f.restype = ctypes.c_size_t
    f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    for path in (0, 1, 2, 3):
        for k in (1, 5, 20, 100, 200, 1000):
            if k > ns:
                continue
            prev = 0
            for nq in list(range(1, 600)) + [1023, 1024, 1025, 4096]:
                w = f(nq, ns, d, k, path)
                assert w >= prev, (path, k, nq)
                prev = w


def test_packed_path_limits_in_workspace_sizes(lib):
    """The packed tensor-core path takes d <= 768 with an even number of
    64-bit words per bitplane and k <= 256: outside those it needs no
    workspace (a call is refused), inside it needs one pass's lists, the
    same for every batch size, and the automatic path's bound covers it
    from four queries up."""
    f = lib.ternary_knn_path_workspace
    f.restype = ctypes.c_size_t
    f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    ns = 1_000_000
    for d in (65, 128, 384, 512, 768):              # W = 2, 2, 6, 8, 12
        w = [f(nq, ns, d, 100, 3) for nq in (1, 16, 64, 65, 300)]
        assert w[0] > 0 and len(set(w)) == 1, (d, w)
        assert f(16, ns, d, 256, 3) > 0
        assert f(16, ns, d, 257, 3) == 0
        for nq in (4, 16, 64):
            assert f(nq, ns, d, 100, 0) >= w[0]
    for d in (64, 129, 700, 1024):                  # W = 1, 3, 11, 16
        assert f(16, ns, d, 100, 3) == 0, d
