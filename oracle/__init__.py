"""EVP oracle: plain, slow CPU reference for the GPU hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The product library never calls it and shares no code with it.

Each function follows a passage of the paper (arXiv 2506.00528):

* ``default_x``  -- Sec. 5.1.1, choice of x maximising C(d, x) * 2^x.
* ``encode``     -- Sec. 2.4, nearest {x,d} vertex: top-x |u_i|, then sign.
* ``pack``/``unpack`` -- Sec. 5.1.2 and Table 3, the v+ / v- bitplanes.
* ``dot``        -- Sec. 5.1.2, b2sp = scalar product of ternary vectors.
* ``delta``      -- notation table and Sec. 2.6: Delta read as squared
  Euclidean distance between ternary vectors (= 2x - 2*b2sp).
* ``knn``        -- Sec. 5.3 / Table 5: exhaustive kNN, (Delta, index) order.
* ``rerank``     -- Sec. 5.3: re-order an n-long shortlist by the original
  float vectors (double-precision scalar product), keep the best k.
* ``quantize_i8`` -- Sec. 6 (single-operand translation): the query kept as
  int8 by symmetric per-query scaling (a reading; the paper fixes no
  precision for the untranslated operand).
* ``masked_sum`` / ``knn_i8q`` -- Sec. 5.1.2 masked addition of a query over
  a ternary code; exhaustive search by that score (largest first).
* ``sparse_pack``/``sparse_unpack`` -- Sec. 6 ("different EVPs"): a code with
  few non-zeros stored as the list of its non-zero dimensions.
* ``l2_knn``     -- the float32 "Euclidean" brute force the paper's speed
  tables compare against (Tables 4 and 5); a CPU baseline, not the method.

The arithmetic lives in ``evp_oracle.c`` (C99, single thread); this module
only marshals numpy arrays.  ``build()`` compiles it with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

_i64 = ctypes.c_int64
_i32 = ctypes.c_int
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile ``evp_oracle.c`` into ``liboracle.so`` (gcc, -O2, C99)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC",
                        _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.evpo_default_x.restype = _i32
            lib.evpo_default_x.argtypes = [_i32]
            lib.evpo_words.restype = _i32
            lib.evpo_words.argtypes = [_i32]
            lib.evpo_encode.restype = _i32
            lib.evpo_encode.argtypes = [_p, _i64, _i32, _i32, _p]
            lib.evpo_pack.restype = None
            lib.evpo_pack.argtypes = [_p, _i64, _i32, _p]
            lib.evpo_unpack.restype = _i64
            lib.evpo_unpack.argtypes = [_p, _i64, _i32, _p]
            lib.evpo_dot.restype = _i64
            lib.evpo_dot.argtypes = [_p, _p, _i32]
            lib.evpo_delta.restype = _i64
            lib.evpo_delta.argtypes = [_p, _p, _i32]
            lib.evpo_knn.restype = _i32
            lib.evpo_knn.argtypes = [_p, _i64, _p, _i64, _i32, _i32, _p, _p]
            lib.evpo_rerank.restype = _i32
            lib.evpo_rerank.argtypes = [_p, _i64, _p, _i64, _i32, _p, _i32, _i32,
                                        _p, _p, _p]
            lib.evpo_quantize_i8.restype = _i32
            lib.evpo_quantize_i8.argtypes = [_p, _i64, _i32, _p]
            lib.evpo_masked_sum.restype = _i64
            lib.evpo_masked_sum.argtypes = [_p, _p, _i32]
            lib.evpo_knn_i8q.restype = _i32
            lib.evpo_knn_i8q.argtypes = [_p, _i64, _p, _i64, _i32, _i32, _p, _p]
            lib.evpo_sparse_pack.restype = _i64
            lib.evpo_sparse_pack.argtypes = [_p, _i64, _i32, _i32, _p]
            lib.evpo_sparse_unpack.restype = _i64
            lib.evpo_sparse_unpack.argtypes = [_p, _i64, _i32, _i32, _p]
            lib.evpo_l2_knn.restype = _i32
            lib.evpo_l2_knn.argtypes = [_p, _i64, _p, _i64, _i32, _i32, _p, _p]
            _lib = lib
    return _lib


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_x(d: int) -> int:
    """Smallest x maximising the {x,d} vertex count C(d,x)*2^x (Sec. 5.1.1)."""
    return int(_load().evpo_default_x(int(d)))


def words(d: int) -> int:
    """64-bit words per bitplane: ceil(d / 64)."""
    return int(_load().evpo_words(int(d)))


class NonFiniteInput(ValueError):
    pass


def encode(U: np.ndarray, x: int, allow_nonfinite: bool = False) -> np.ndarray:
    """Nearest {x,d} EVP vertex of each row of U (Sec. 2.4) as int8 [n, d]."""
    U = _c(U, np.float32)
    if U.ndim != 2:
        raise ValueError("U must be 2-D [n, d]")
    n, d = U.shape
    if not 1 <= x <= d:
        raise ValueError("x must satisfy 1 <= x <= d")
    V = np.zeros((n, d), dtype=np.int8)
    rc = _load().evpo_encode(_ptr(U), n, d, int(x), _ptr(V))
    if rc < 0:
        raise MemoryError("oracle encode allocation failed")
    if rc and not allow_nonfinite:
        raise NonFiniteInput("non-finite value in input rows")
    return V


def pack(V: np.ndarray) -> np.ndarray:
    """Ternary int8 [n, d] -> bitplanes uint64 [n, 2W] (v+ words, then v-)."""
    V = _c(V, np.int8)
    n, d = V.shape
    W = words(d)
    T = np.zeros((n, 2 * W), dtype=np.uint64)
    _load().evpo_pack(_ptr(V), n, d, _ptr(T))
    return T


def unpack(T: np.ndarray, d: int) -> tuple[np.ndarray, int]:
    """Bitplanes -> ternary int8 [n, d]; also the number of malformed rows."""
    T = _c(T, np.uint64)
    n = T.shape[0]
    if T.shape[1] != 2 * words(d):
        raise ValueError("bitplane width does not match d")
    V = np.zeros((n, d), dtype=np.int8)
    bad = _load().evpo_unpack(_ptr(T), n, int(d), _ptr(V))
    return V, int(bad)


def dot(v: np.ndarray, w: np.ndarray) -> int:
    """b2sp(v, w): scalar product of two ternary vectors (Sec. 5.1.2)."""
    v = _c(v, np.int8).ravel()
    w = _c(w, np.int8).ravel()
    assert v.size == w.size
    return int(_load().evpo_dot(_ptr(v), _ptr(w), v.size))


def delta(v: np.ndarray, w: np.ndarray) -> int:
    """Delta(v, w) = ||v - w||^2 over ternary vectors."""
    v = _c(v, np.int8).ravel()
    w = _c(w, np.int8).ravel()
    assert v.size == w.size
    return int(_load().evpo_delta(_ptr(v), _ptr(w), v.size))


def knn(Vq: np.ndarray, Vs: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Exhaustive kNN by Delta with (Delta, index) order: ids int64, dist int32."""
    Vq = _c(Vq, np.int8)
    Vs = _c(Vs, np.int8)
    nq, d = Vq.shape
    ns, d2 = Vs.shape
    assert d == d2
    if not 1 <= k <= ns:
        raise ValueError("k must satisfy 1 <= k <= ns")
    ids = np.zeros((nq, k), dtype=np.int64)
    dist = np.zeros((nq, k), dtype=np.int32)
    rc = _load().evpo_knn(_ptr(Vq), nq, _ptr(Vs), ns, d, int(k), _ptr(ids), _ptr(dist))
    if rc != 0:
        raise MemoryError("oracle knn failed")
    return ids, dist


def rerank(Q: np.ndarray, S: np.ndarray, shortlist: np.ndarray, k: int):
    """Re-order each query's shortlist by <q, s> in float64 (Sec. 5.3).

    Returns (ids int64 [nq, k], scores float64 [nq, k], absdot float64 [nq, k]).
    """
    Q = _c(Q, np.float32)
    S = _c(S, np.float32)
    sl = _c(shortlist, np.int64)
    nq, d = Q.shape
    ns = S.shape[0]
    n = sl.shape[1]
    ids = np.zeros((nq, k), dtype=np.int64)
    scores = np.zeros((nq, k), dtype=np.float64)
    absdot = np.zeros((nq, k), dtype=np.float64)
    rc = _load().evpo_rerank(_ptr(Q), nq, _ptr(S), ns, d, _ptr(sl), int(n), int(k),
                             _ptr(ids), _ptr(scores), _ptr(absdot))
    if rc != 0:
        raise ValueError("shortlist id out of range")
    return ids, scores, absdot


def quantize_i8(Q: np.ndarray, allow_nonfinite: bool = False) -> np.ndarray:
    """Per-query symmetric int8 quantisation (Sec. 6 reading): float32 [n, d] -> int8."""
    Q = _c(Q, np.float32)
    n, d = Q.shape
    out = np.zeros((n, d), dtype=np.int8)
    bad = _load().evpo_quantize_i8(_ptr(Q), n, d, _ptr(out))
    if bad and not allow_nonfinite:
        raise NonFiniteInput("non-finite value in query rows")
    return out


def masked_sum(q8: np.ndarray, v: np.ndarray) -> int:
    """Masked addition (Sec. 5.1.2): sum of q8 where v = +1 minus where v = -1."""
    q8 = _c(q8, np.int8).ravel()
    v = _c(v, np.int8).ravel()
    assert q8.size == v.size
    return int(_load().evpo_masked_sum(_ptr(q8), _ptr(v), q8.size))


def knn_i8q(Q8: np.ndarray, Vs: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Exhaustive search by masked-addition score: ids int64, score int32 [nq, k],
    largest score first, equal scores by lower index."""
    Q8 = _c(Q8, np.int8)
    Vs = _c(Vs, np.int8)
    nq, d = Q8.shape
    ns = Vs.shape[0]
    assert Vs.shape[1] == d
    if not 1 <= k <= ns:
        raise ValueError("k must satisfy 1 <= k <= ns")
    ids = np.zeros((nq, k), dtype=np.int64)
    score = np.zeros((nq, k), dtype=np.int32)
    if _load().evpo_knn_i8q(_ptr(Q8), nq, _ptr(Vs), ns, d, int(k), _ptr(ids), _ptr(score)):
        raise MemoryError("oracle knn_i8q failed")
    return ids, score


def sparse_pack(V: np.ndarray, x: int) -> np.ndarray:
    """Ternary int8 [n, d] with x non-zeros per row -> uint16 [n, x] index lists
    (bit 15 = -1, bits 0-14 = dimension, ascending)."""
    V = _c(V, np.int8)
    n, d = V.shape
    E = np.zeros((n, int(x)), dtype=np.uint16)
    bad = _load().evpo_sparse_pack(_ptr(V), n, d, int(x), _ptr(E))
    if bad:
        raise ValueError(f"{bad} rows do not have exactly x non-zeros")
    return E


def sparse_unpack(E: np.ndarray, d: int) -> tuple[np.ndarray, int]:
    """Index lists uint16 [n, x] -> ternary int8 [n, d]; also the number of
    malformed rows."""
    E = _c(E, np.uint16)
    n, x = E.shape
    V = np.zeros((n, int(d)), dtype=np.int8)
    bad = _load().evpo_sparse_unpack(_ptr(E), n, int(d), int(x), _ptr(V))
    return V, int(bad)


def l2_knn(Q: np.ndarray, S: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Float32 exhaustive kNN by squared Euclidean distance (the paper's
    "Euclidean" speed baseline): ids int64, dist float32 [nq, k]."""
    Q = _c(Q, np.float32)
    S = _c(S, np.float32)
    nq, d = Q.shape
    ns = S.shape[0]
    ids = np.zeros((nq, k), dtype=np.int64)
    dist = np.zeros((nq, k), dtype=np.float32)
    if _load().evpo_l2_knn(_ptr(Q), nq, _ptr(S), ns, d, int(k), _ptr(ids), _ptr(dist)):
        raise ValueError("oracle l2_knn failed")
    return ids, dist
