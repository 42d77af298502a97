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

PATH_AUTO, PATH_POPC, PATH_MMA, PATH_MMA_PACKED = 0, 1, 2, 3
MMA_MAX_K = 1024

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
    "ternary_knn_path_workspace": (_sz, [_i64, _i64, _i32, _i32, _i32]),
    "ternary_knn_path": (_i32, [_p, _i64, _p, _i64, _i32, _i32, _i32, _p, _p, _p, _sz, _p, _p,
                                _i32]),
    "ternary_knn_static": (_i32, [_p, _i64, _p, _i64, _i32, _i32, _i32, _p, _p, _p, _p]),
    "evp_quantize_i8": (_i32, [_p, _i64, _i32, _p, _p, _p]),
    "evp_pack_sparse": (_i32, [_p, _i64, _i32, _i32, _p, _p, _p]),
    "ternary_knn_sparse_workspace": (_sz, [_i64, _i64, _i32, _i32, _i32]),
    "ternary_knn_sparse": (_i32, [_p, _i64, _p, _i64, _i32, _i32, _i32, _p, _p, _p, _sz, _p, _p]),
    "ternary_knn_i8q_workspace": (_sz, [_i64, _i64, _i32, _i32]),
    "ternary_knn_i8q": (_i32, [_p, _i64, _p, _i64, _i32, _i32, _i32, _p, _p, _p, _sz, _p, _p]),
    "rerank": (_i32, [_p, _i64, _p, _i64, _i32, _p, _i32, _i32, _p, _p, _p, _p]),
    "evp_merge_topk_workspace": (_sz, [_i64, _i32, _i32]),
    "evp_merge_topk": (_i32, [_p, _p, _i64, _i32, _i32, _p, _p, _p, _sz, _p, _p]),
    "evp_db_create": (_i32, [_p, _p, _i64, _i32, _i32, _i32, _p, ctypes.POINTER(_p)]),
    "evp_db_destroy": (_i32, [_p]),
    "evp_db_knn_workspace": (_sz, [_p, _i64, _i32, _i32]),
    "evp_db_knn": (_i32, [_p, _p, _i64, _i32, _p, _p, _p, _sz, _p, _p, _i32]),
    "evp_db_search_workspace": (_sz, [_p, _i64, _i32, _i32]),
    "evp_db_search": (_i32, [_p, _p, _i64, _i32, _i32, _p, _p, _p, _sz, _p, _p]),
    "evp_db_search_host_workspace": (_sz, [_p, _i64, _i32, _i32]),
    "evp_db_search_host": (_i32, [_p, _p, _i64, _i32, _i32, _p, _p, _p, _sz, _p, _p]),
    "evp_db_dim": (_i32, [_p]),
    "evp_db_rows": (_i64, [_p]),
    "evp_server_create": (_i32, [_p, _p, ctypes.POINTER(_p)]),
    "evp_server_slots": (_i32, [_p]),
    "evp_server_submit": (_i32, [_p, _p, _i64, _i32, _p, _p, ctypes.POINTER(_i64)]),
    "evp_server_wait": (_i32, [_p, _i64, _i64, ctypes.POINTER(_i32),
                               ctypes.POINTER(ctypes.c_double)]),
    "evp_server_stats": (_i32, [_p, _p]),
    "evp_server_reset_stats": (_i32, [_p]),
    "evp_server_pause": (_i32, [_p, _i32]),
    "evp_server_destroy": (_i32, [_p]),
    "evp_db_codes": (_p, [_p]),
    "evp_db_search_path_workspace": (_sz, [_p, _i64, _i32, _i32, _i32]),
    "evp_db_search_path": (_i32, [_p, _p, _i64, _i32, _i32, _p, _p, _p, _sz, _p, _p, _i32]),
    "evp_autotune": (_i32, [_p, _i64, _i32, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float),
                            ctypes.POINTER(ctypes.c_float), _p]),
    "evp_autotune_clear": (_i32, []),
    "evp_autotune_save": (_i32, [ctypes.c_char_p]),
    "evp_autotune_load": (_i32, [ctypes.c_char_p]),
    "evp_batch_plan_fused": (_i32, [_p]),
    "evp_batch_plan_tile": (_i32, [_p, _i32]),
    "evp_batch_plan_create": (_i32, [_p, _i32, _i32, _p, ctypes.POINTER(_p)]),
    "evp_batch_plan_path": (_i32, [_p, _i32]),
    "evp_batch_plan_workspace": (_sz, [_p]),
    "evp_batch_run": (_i32, [_p, _p, _p]),
    "evp_batch_plan_destroy": (_i32, [_p]),
    "evp_test_stall_producer": (_i32, [_i32, _i32]),
    "evp_probe_tensor_rate": (_i32, [_i32, _i32, _i32, _i64, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), _p]),
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


def knn_workspace_bytes(nq: int, ns: int, d: int, k: int, path: int = PATH_AUTO) -> int:
    return int(load().ternary_knn_path_workspace(int(nq), int(ns), int(d), int(k), int(path)))


def ternary_knn(Q: torch.Tensor, S: torch.Tensor, d: int, x: int, k: int,
                ids: torch.Tensor | None = None, dist: torch.Tensor | None = None,
                ws: torch.Tensor | None = None, status: torch.Tensor | None = None,
                stream=None, path: int = PATH_AUTO):
    """ternary_knn: packed Q [nq, 2W], packed S [ns, 2W] -> ids int64, dist int32 [nq, k]."""
    _req(Q, torch.int64, "Q")
    _req(S, torch.int64, "S")
    nq, ns = Q.shape[0], S.shape[0]
    if ids is None:
        ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
    if dist is None:
        dist = torch.empty((nq, k), dtype=torch.int32, device=Q.device)
    need = knn_workspace_bytes(nq, ns, d, k, path)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=Q.device)
    if path == PATH_AUTO:
        rc = load().ternary_knn(_ptr(Q), nq, _ptr(S), ns, int(d), int(x), int(k), _ptr(ids),
                                _ptr(dist), _ptr(ws), ws.numel(), _ptr(status),
                                _stream_handle(stream))
    else:
        rc = load().ternary_knn_path(_ptr(Q), nq, _ptr(S), ns, int(d), int(x), int(k),
                                     _ptr(ids), _ptr(dist), _ptr(ws), ws.numel(), _ptr(status),
                                     _stream_handle(stream), int(path))
    _check(rc, "ternary_knn")
    return ids, dist


def quantize_i8(Q: torch.Tensor, out: torch.Tensor | None = None,
                status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """evp_quantize_i8: float32 [nq, d] -> int8 [nq, d] (symmetric per query)."""
    _req(Q, torch.float32, "Q")
    nq, d = Q.shape
    if out is None:
        out = torch.empty((nq, d), dtype=torch.int8, device=Q.device)
    _req(out, torch.int8, "out")
    if tuple(out.shape) != (nq, d):
        raise ValueError("out must have the shape of Q")
    _check(load().evp_quantize_i8(_ptr(Q), nq, d, _ptr(out), _ptr(status), _stream_handle(stream)),
           "evp_quantize_i8")
    return out


def ternary_knn_i8q(Q8: torch.Tensor, S: torch.Tensor, d: int, x: int, k: int,
                    ids: torch.Tensor | None = None, score: torch.Tensor | None = None,
                    ws: torch.Tensor | None = None, status: torch.Tensor | None = None,
                    stream=None):
    """ternary_knn_i8q: int8 queries [nq, d], packed S [ns, 2W] -> ids int64,
    score int32 [nq, k] (largest masked-addition score first)."""
    _req(Q8, torch.int8, "Q8")
    _req(S, torch.int64, "S")
    nq, ns = Q8.shape[0], S.shape[0]
    if Q8.shape[1] != d or S.shape[1] != 2 * words(d):
        raise ValueError("Q8 must be [nq, d] and S [ns, 2W]")
    if ids is None:
        ids = torch.empty((nq, k), dtype=torch.int64, device=Q8.device)
    if score is None:
        score = torch.empty((nq, k), dtype=torch.int32, device=Q8.device)
    need = int(load().ternary_knn_i8q_workspace(nq, ns, int(d), int(k)))
    if need == 0:
        raise EvpError(EVP_ERR_UNSUPPORTED, "ternary_knn_i8q")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=Q8.device)
    _check(load().ternary_knn_i8q(_ptr(Q8), nq, _ptr(S), ns, int(d), int(x), int(k), _ptr(ids),
                                  _ptr(score), _ptr(ws), ws.numel(), _ptr(status),
                                  _stream_handle(stream)), "ternary_knn_i8q")
    return ids, score


def pack_sparse(T: torch.Tensor, d: int, x: int, out: torch.Tensor | None = None,
                status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """evp_pack_sparse: packed codes [n, 2W] -> sparse codes int16 [n, x]
    (the uint16 entries' bits: dimension | 0x8000 for -1)."""
    _req(T, torch.int64, "T")
    n = T.shape[0]
    if T.shape[1] != 2 * words(d):
        raise ValueError("T must be [n, 2W] packed codes for this d")
    if out is None:
        out = torch.empty((n, int(x)), dtype=torch.int16, device=T.device)
    _req(out, torch.int16, "out")
    if tuple(out.shape) != (n, int(x)):
        raise ValueError("out must be [n, x]")
    _check(load().evp_pack_sparse(_ptr(T), n, int(d), int(x), _ptr(out), _ptr(status),
                                  _stream_handle(stream)), "evp_pack_sparse")
    return out


def ternary_knn_sparse(Q: torch.Tensor, E: torch.Tensor, d: int, x: int, k: int,
                       ids: torch.Tensor | None = None, dist: torch.Tensor | None = None,
                       ws: torch.Tensor | None = None, status: torch.Tensor | None = None,
                       stream=None):
    """ternary_knn_sparse: packed queries [nq, 2W], sparse database [ns, x]
    -> ids int64, dist int32 [nq, k] (the results of ternary_knn)."""
    _req(Q, torch.int64, "Q")
    _req(E, torch.int16, "E")
    nq, ns = Q.shape[0], E.shape[0]
    if Q.shape[1] != 2 * words(d) or E.shape[1] != x:
        raise ValueError("Q must be [nq, 2W] and E [ns, x]")
    if ids is None:
        ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
    if dist is None:
        dist = torch.empty((nq, k), dtype=torch.int32, device=Q.device)
    need = int(load().ternary_knn_sparse_workspace(nq, ns, int(d), int(x), int(k)))
    if need == 0:
        raise EvpError(EVP_ERR_UNSUPPORTED, "ternary_knn_sparse")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=Q.device)
    _check(load().ternary_knn_sparse(_ptr(Q), nq, _ptr(E), ns, int(d), int(x), int(k), _ptr(ids),
                                     _ptr(dist), _ptr(ws), ws.numel(), _ptr(status),
                                     _stream_handle(stream)), "ternary_knn_sparse")
    return ids, dist


def ternary_knn_static(Q: torch.Tensor, S: torch.Tensor, d: int, x: int, k: int,
                       ids: torch.Tensor, dist: torch.Tensor, status: torch.Tensor | None = None,
                       stream=None):
    """ternary_knn_static: the popcount scan with the library's fixed scratch
    (no allocation by the library; outputs must be given)."""
    _req(Q, torch.int64, "Q")
    _req(S, torch.int64, "S")
    _req(ids, torch.int64, "ids")
    _req(dist, torch.int32, "dist")
    nq = Q.shape[0]
    if Q.dim() != 2 or S.dim() != 2 or Q.shape[1] != 2 * words(d) or S.shape[1] != Q.shape[1]:
        raise ValueError("Q and S must be [n, 2W] packed codes for this d")
    if tuple(ids.shape) != (nq, int(k)) or tuple(dist.shape) != (nq, int(k)):
        raise ValueError(f"ids and dist must both have shape ({nq}, {int(k)})")
    if len({Q.device, S.device, ids.device, dist.device}) != 1:
        raise ValueError("Q, S, ids and dist must be on the same device")
    rc = load().ternary_knn_static(_ptr(Q), Q.shape[0], _ptr(S), S.shape[0], int(d), int(x),
                                   int(k), _ptr(ids), _ptr(dist), _ptr(status),
                                   _stream_handle(stream))
    _check(rc, "ternary_knn_static")
    return ids, dist


def merge_topk(ids: torch.Tensor, dist: torch.Tensor, k: int, status=None, stream=None):
    """evp_merge_topk: per-shard results ids/dist [nlists, nq, k] -> global top-k [nq, k]."""
    _req(ids, torch.int64, "ids")
    _req(dist, torch.int32, "dist")
    nlists, nq = ids.shape[0], ids.shape[1]
    out_i = torch.empty((nq, k), dtype=torch.int64, device=ids.device)
    out_d = torch.empty((nq, k), dtype=torch.int32, device=ids.device)
    need = int(load().evp_merge_topk_workspace(nq, nlists, int(k)))
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=ids.device)
    _check(load().evp_merge_topk(_ptr(ids), _ptr(dist), nq, nlists, int(k), _ptr(out_i),
                                 _ptr(out_d), _ptr(ws), ws.numel(), _ptr(status),
                                 _stream_handle(stream)), "evp_merge_topk")
    return out_i, out_d


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


def test_stall_producer(path: int, fills: int):
    """Testing support: the next launch of the tensor-core scan `path` stalls
    its first CTA's copy producer after `fills` stage fills (evp.h)."""
    _check(load().evp_test_stall_producer(int(path), int(fills)), "evp_test_stall_producer")


def probe_tensor_rate(kind: int = 0, cta_pair: bool = False, n: int = 256,
                      iters: int = 1 << 16, stream=None):
    """evp_probe_tensor_rate: (TFLOP/s, SM clocks per instruction, ms) of
    back-to-back tcgen05.mma (kind 0 = e4m3 f8f6f4, 1 = bf16 f16) on every SM.
    kind | 0x100 / 0x200: zero / random operands; | 0x400: A in tensor memory;
    | 0x800: M = 64."""
    tf, cyc, ms = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    _check(load().evp_probe_tensor_rate(int(kind), 1 if cta_pair else 0, int(n), int(iters),
                                        ctypes.byref(tf), ctypes.byref(cyc), ctypes.byref(ms),
                                        _stream_handle(stream)), "evp_probe_tensor_rate")
    return tf.value, cyc.value, ms.value


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


class Database:
    """Resident database handle (evp_db_*): packed codes T [ns, 2W] (int64
    bits) and optional float rows U [ns, d] stay on the device; the handle
    keeps references to both so they outlive it."""

    def __init__(self, T: torch.Tensor, U: torch.Tensor | None, d: int, x: int,
                 tensor_copy: bool = True, stream=None):
        _req(T, torch.int64, "T")
        if U is not None:
            _req(U, torch.float32, "U")
        self.T, self.U, self.d, self.x = T, U, int(d), int(x)
        self.ns = T.shape[0]
        h = ctypes.c_void_p()
        rc = load().evp_db_create(_ptr(T), _ptr(U), self.ns, self.d, self.x,
                                  1 if tensor_copy else 0, _stream_handle(stream), ctypes.byref(h))
        _check(rc, "evp_db_create")
        self.handle = h
        self._ws = None

    def close(self):
        if getattr(self, "handle", None):
            _check(load().evp_db_destroy(self.handle), "evp_db_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _workspace(self, need: int, ws):
        if ws is not None and ws.numel() >= need:
            return ws
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.T.device)
        return self._ws

    def knn(self, Q: torch.Tensor, k: int, ids=None, dist=None, ws=None, status=None,
            stream=None, path: int = PATH_AUTO):
        _req(Q, torch.int64, "Q")
        nq = Q.shape[0]
        ids = ids if ids is not None else torch.empty((nq, k), dtype=torch.int64, device=Q.device)
        dist = dist if dist is not None else torch.empty((nq, k), dtype=torch.int32, device=Q.device)
        need = int(load().evp_db_knn_workspace(self.handle, nq, int(k), int(path)))
        ws = self._workspace(need, ws)
        rc = load().evp_db_knn(self.handle, _ptr(Q), nq, int(k), _ptr(ids), _ptr(dist),
                               _ptr(ws), ws.numel(), _ptr(status), _stream_handle(stream),
                               int(path))
        _check(rc, "evp_db_knn")
        return ids, dist

    def search_workspace_bytes(self, nq: int, n_shortlist: int, k: int) -> int:
        return int(load().evp_db_search_workspace(self.handle, nq, int(n_shortlist), int(k)))

    def search(self, Q: torch.Tensor, n_shortlist: int, k: int, ids=None, scores=None, ws=None,
               status=None, stream=None):
        """encode -> scan (n_shortlist by Delta) -> rerank (k by <q, s>)."""
        _req(Q, torch.float32, "Q")
        nq = Q.shape[0]
        ids = ids if ids is not None else torch.empty((nq, k), dtype=torch.int64, device=Q.device)
        scores = scores if scores is not None else torch.empty((nq, k), dtype=torch.float32,
                                                               device=Q.device)
        ws = self._workspace(self.search_workspace_bytes(nq, n_shortlist, k), ws)
        rc = load().evp_db_search(self.handle, _ptr(Q), nq, int(n_shortlist), int(k), _ptr(ids),
                                  _ptr(scores), _ptr(ws), ws.numel(), _ptr(status),
                                  _stream_handle(stream))
        _check(rc, "evp_db_search")
        return ids, scores

    def search_host_workspace_bytes(self, nq: int, n_shortlist: int, k: int) -> int:
        return int(load().evp_db_search_host_workspace(self.handle, nq, int(n_shortlist), int(k)))

    def search_host(self, Q_host: torch.Tensor, n_shortlist: int, k: int, ids_host: torch.Tensor,
                    scores_host: torch.Tensor, ws=None, status=None, stream=None):
        """The same path with host (preferably pinned) buffers; asynchronous."""
        if Q_host.is_cuda or Q_host.dtype != torch.float32 or not Q_host.is_contiguous():
            raise ValueError("Q_host must be a contiguous host float32 tensor")
        nq = Q_host.shape[0]
        ws = self._workspace(self.search_host_workspace_bytes(nq, n_shortlist, k), ws)
        rc = load().evp_db_search_host(self.handle, _ptr(Q_host), nq, int(n_shortlist), int(k),
                                       _ptr(ids_host), _ptr(scores_host), _ptr(ws), ws.numel(),
                                       _ptr(status), _stream_handle(stream))
        _check(rc, "evp_db_search_host")


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_batch_queries", ctypes.c_int32),
                ("max_k", ctypes.c_int32), ("shortlist_factor", ctypes.c_int32),
                ("max_slots", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_int64), ("queries", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("max_us", ctypes.c_double)]


class Server:
    """Continuous-batching request loop (evp_server_*) over a Database."""

    def __init__(self, db: "Database", max_batch_queries: int = 1024, max_k: int = 100,
                 shortlist_factor: int = 10, max_slots: int = 3, mem_budget_bytes: int = 0,
                 device: int | None = None):
        self.db = db
        cfg = ServerConfig(device if device is not None else db.T.device.index or 0,
                           max_batch_queries, max_k, shortlist_factor, max_slots,
                           mem_budget_bytes)
        h = ctypes.c_void_p()
        _check(load().evp_server_create(db.handle, ctypes.byref(cfg), ctypes.byref(h)),
               "evp_server_create")
        self.handle = h
        self._live = {}

    @property
    def slots(self) -> int:
        return int(load().evp_server_slots(self.handle))

    def submit(self, Q_host, k: int) -> int:
        """Queue float32 host queries [nq, d]; returns a request id."""
        Q = torch.as_tensor(Q_host)
        if Q.is_cuda or Q.dtype != torch.float32 or not Q.is_contiguous():
            raise ValueError("Q_host must be a contiguous host float32 tensor or array")
        nq = Q.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int64)
        sc = torch.empty((nq, k), dtype=torch.float32)
        rid = ctypes.c_int64(0)
        _check(load().evp_server_submit(self.handle, _ptr(Q), nq, int(k), _ptr(ids), _ptr(sc),
                                        ctypes.byref(rid)), "evp_server_submit")
        self._live[rid.value] = (Q, ids, sc)
        return int(rid.value)

    def wait(self, rid: int, timeout_s: float = 30.0):
        """(ids, scores, status, latency_us); raises EvpError(EVP_ERR_TIMEOUT) on timeout."""
        st = ctypes.c_int32(0)
        lat = ctypes.c_double(0.0)
        _check(load().evp_server_wait(self.handle, int(rid), int(timeout_s * 1e6),
                                      ctypes.byref(st), ctypes.byref(lat)), "evp_server_wait")
        _, ids, sc = self._live.pop(int(rid))
        return ids, sc, int(st.value), float(lat.value)

    def pause(self, paused: bool = True):
        _check(load().evp_server_pause(self.handle, 1 if paused else 0), "evp_server_pause")

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().evp_server_stats(self.handle, ctypes.byref(s)), "evp_server_stats")
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def reset_stats(self):
        _check(load().evp_server_reset_stats(self.handle), "evp_server_reset_stats")

    def close(self):
        if getattr(self, "handle", None):
            _check(load().evp_server_destroy(self.handle), "evp_server_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchDesc(ctypes.Structure):
    _fields_ = [("db", ctypes.c_void_p), ("Q", ctypes.c_void_p), ("Qc", ctypes.c_void_p),
                ("nq", ctypes.c_int64), ("n_shortlist", ctypes.c_int32), ("k", ctypes.c_int32),
                ("ids", ctypes.c_void_p), ("scores", ctypes.c_void_p), ("dist", ctypes.c_void_p)]


def autotune(db: "Database", nq: int, k: int, measure: bool = False, stream=None):
    """(path, popc_ms, mma_ms) from evp_autotune (timings only when measured)."""
    path = ctypes.c_int32(0)
    pm, mm = ctypes.c_float(0.0), ctypes.c_float(0.0)
    args = (ctypes.byref(pm), ctypes.byref(mm)) if measure else (None, None)
    _check(load().evp_autotune(db.handle, int(nq), int(k), ctypes.byref(path), *args,
                               _stream_handle(stream)), "evp_autotune")
    return int(path.value), (pm.value if measure else None), (mm.value if measure else None)


def autotune_save(path: str):
    _check(load().evp_autotune_save(path.encode()), "evp_autotune_save")


def autotune_load(path: str):
    _check(load().evp_autotune_load(path.encode()), "evp_autotune_load")


class BatchPlan:
    """evp_batch_plan_*: a list of search / kNN batches planned once and run
    (optionally as one captured CUDA graph).  Each item of `batches` is a dict
    with db, and either Q (float32 [nq, d]) + n_shortlist + k (search) or Qc
    (packed codes) + k (kNN); outputs are allocated here."""

    def __init__(self, batches, graph: bool = True, tune: bool = True, stream=None,
                 fused: bool = True):
        self.items = []
        descs = (BatchDesc * len(batches))()
        for i, b in enumerate(batches):
            db = b["db"]
            k = int(b["k"])
            if b.get("Q") is not None:
                Q = b["Q"]
                _req(Q, torch.float32, "Q")
                nq = Q.shape[0]
                ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
                sc = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
                descs[i] = BatchDesc(db.handle, _ptr(Q), None, nq, int(b["n_shortlist"]), k,
                                     _ptr(ids), _ptr(sc), None)
                self.items.append((Q, ids, sc))
            else:
                Qc = b["Qc"]
                _req(Qc, torch.int64, "Qc")
                nq = Qc.shape[0]
                ids = torch.empty((nq, k), dtype=torch.int64, device=Qc.device)
                dist = torch.empty((nq, k), dtype=torch.int32, device=Qc.device)
                descs[i] = BatchDesc(db.handle, None, _ptr(Qc), nq, 0, k, _ptr(ids), None,
                                     _ptr(dist))
                self.items.append((Qc, ids, dist))
        self.dbs = [b["db"] for b in batches]
        flags = (1 if graph else 0) | (0 if tune else 2) | (0 if fused else 4)
        h = ctypes.c_void_p()
        _check(load().evp_batch_plan_create(descs, len(batches), flags, _stream_handle(stream),
                                            ctypes.byref(h)), "evp_batch_plan_create")
        self.handle = h
        self._descs = descs

    def path(self, i: int) -> int:
        return int(load().evp_batch_plan_path(self.handle, int(i)))

    @property
    def fused(self) -> int:
        """Batches scanned by the fused launch."""
        return int(load().evp_batch_plan_fused(self.handle))

    def tile(self, i: int) -> int:
        return int(load().evp_batch_plan_tile(self.handle, int(i)))

    def run(self, status=None, stream=None):
        _check(load().evp_batch_run(self.handle, _ptr(status), _stream_handle(stream)),
               "evp_batch_run")

    def outputs(self, i: int):
        return self.items[i][1], self.items[i][2]

    def close(self):
        if getattr(self, "handle", None):
            _check(load().evp_batch_plan_destroy(self.handle), "evp_batch_plan_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
