"""Thin ctypes binding of libevp (include/evp.h) for torch CUDA tensors.

Argument marshalling only: every step of the path runs in the library's
CUDA kernels.  Torch provides device memory and streams.  Packed codes are
held in torch.int64 tensors of shape [n, 2W] whose bits are the uint64
words of the boundary format (v+ words, then v- words).

If libevp.so has not been built the first call raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libevp.so")

EVP_OK = 0
EVP_ERR_INVALID = 1
EVP_ERR_NONFINITE = 2
EVP_ERR_NO_MEMORY = 3
EVP_ERR_TIMEOUT = 4
EVP_ERR_CUDA = 5
EVP_ERR_UNSUPPORTED = 6
EVP_ERR_RANGE = 7

MAX_D_ENCODE = 2048
MAX_D_SCAN = 1024
MAX_K = 1024
MAX_SHORTLIST = 4096
MAX_D_RERANK = 4096

_lib = None
_lock = threading.Lock()
_i64, _i32, _p, _sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t

# name -> (restype, argtypes); mirrors include/evp.h
SIGNATURES = {
    "evp_status_string": (ctypes.c_char_p, [_i32]),
    "evp_version": (_i32, []),
    "evp_words": (_i32, [_i32]),
    "evp_default_x": (_i32, [_i32]),
    "evp_encode": (_i32, [_p, _i64, _i32, _i32, _p, _p, _p]),
    "ternary_knn_workspace": (_sz, [_i64, _i64, _i32, _i32]),
    "ternary_knn": (_i32, [_p, _i64, _p, _i64, _i32, _i32, _i32, _p, _p, _p, _sz, _p, _p]),
    "rerank": (_i32, [_p, _i64, _p, _i64, _i32, _p, _i32, _i32, _p, _p, _p, _p]),
    "evp_timing_enable": (_i32, [_i32]),
    "evp_timing_reset": (_i32, []),
    "evp_timing_read": (_i32, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_double)]),
}


class EvpError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = int(code)
        super().__init__(f"{where}: {status_string(code)}" if where else status_string(code))


def load(path: str = LIB_PATH):
    """Load libevp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libevp.so not found at {path}: build it first "
                                   "(python -m paper_2506_00528_gb300.build)")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_string(code: int) -> str:
    return load().evp_status_string(int(code)).decode()


def words(d: int) -> int:
    return int(load().evp_words(int(d)))


def default_x(d: int) -> int:
    return int(load().evp_default_x(int(d)))


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _check(rc: int, where: str):
    if rc != EVP_OK:
        raise EvpError(rc, where)


def new_status(device="cuda") -> torch.Tensor:
    """A zeroed device int32 status word for the dev_status argument."""
    return torch.zeros(1, dtype=torch.int32, device=device)


def check_status(status: torch.Tensor, where: str = "device"):
    """Synchronise on the status word and raise if a kernel reported an error."""
    v = int(status.item())
    if v != EVP_OK:
        raise EvpError(v, where)


def _req(t: torch.Tensor, dtype, name: str):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")


def encode(U: torch.Tensor, x: int, out: torch.Tensor | None = None,
           status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """evp_encode: float32 [n, d] -> packed codes int64 [n, 2W]."""
    _req(U, torch.float32, "U")
    n, d = U.shape
    W = words(d)
    if out is None:
        out = torch.empty((n, 2 * W), dtype=torch.int64, device=U.device)
    rc = load().evp_encode(_ptr(U), n, d, int(x), _ptr(out), _ptr(status), _stream_handle(stream))
    _check(rc, "evp_encode")
    return out


def knn_workspace_bytes(nq: int, ns: int, d: int, k: int) -> int:
    return int(load().ternary_knn_workspace(int(nq), int(ns), int(d), int(k)))


def ternary_knn(Q: torch.Tensor, S: torch.Tensor, d: int, x: int, k: int,
                ids: torch.Tensor | None = None, dist: torch.Tensor | None = None,
                ws: torch.Tensor | None = None, status: torch.Tensor | None = None,
                stream=None):
    """ternary_knn: packed Q [nq, 2W], packed S [ns, 2W] -> ids int64, dist int32 [nq, k]."""
    _req(Q, torch.int64, "Q")
    _req(S, torch.int64, "S")
    nq, ns = Q.shape[0], S.shape[0]
    if ids is None:
        ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
    if dist is None:
        dist = torch.empty((nq, k), dtype=torch.int32, device=Q.device)
    need = knn_workspace_bytes(nq, ns, d, k)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=Q.device)
    rc = load().ternary_knn(_ptr(Q), nq, _ptr(S), ns, int(d), int(x), int(k), _ptr(ids),
                            _ptr(dist), _ptr(ws), ws.numel(), _ptr(status), _stream_handle(stream))
    _check(rc, "ternary_knn")
    return ids, dist


def rerank(Q: torch.Tensor, S: torch.Tensor, shortlist: torch.Tensor, k: int,
           ids: torch.Tensor | None = None, scores: torch.Tensor | None = None,
           status: torch.Tensor | None = None, stream=None):
    """rerank: float Q [nq, d], float S [ns, d], shortlist int64 [nq, n] -> ids, scores [nq, k]."""
    _req(Q, torch.float32, "Q")
    _req(S, torch.float32, "S")
    _req(shortlist, torch.int64, "shortlist")
    nq, d = Q.shape
    n = shortlist.shape[1]
    if ids is None:
        ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
    if scores is None:
        scores = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
    rc = load().rerank(_ptr(Q), nq, _ptr(S), S.shape[0], d, _ptr(shortlist), int(n), int(k),
                       _ptr(ids), _ptr(scores), _ptr(status), _stream_handle(stream))
    _check(rc, "rerank")
    return ids, scores


def timing_enable(on: bool = True):
    _check(load().evp_timing_enable(1 if on else 0), "evp_timing_enable")


def timing_reset():
    _check(load().evp_timing_reset(), "evp_timing_reset")


def timing_read(name: str):
    """(launches, total_ms) of the named kernel family since the last reset."""
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    _check(load().evp_timing_read(name.encode(), ctypes.byref(n), ctypes.byref(ms)),
           "evp_timing_read")
    return int(n.value), float(ms.value)
