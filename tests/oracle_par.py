"""Run oracle calls on row chunks in threads (the C oracle releases the GIL
inside ctypes calls), so large oracle checks use the host's cores."""
import concurrent.futures as cf
import os

import numpy as np

import oracle

THREADS = max(1, min(32, os.cpu_count() or 1))


def encode(U: np.ndarray, x: int) -> np.ndarray:
    n = U.shape[0]
    if n < 4096:
        return oracle.encode(U, x)
    bounds = np.linspace(0, n, THREADS + 1).astype(np.int64)
    out = np.empty(U.shape, dtype=np.int8)

    def job(i):
        a, b = bounds[i], bounds[i + 1]
        out[a:b] = oracle.encode(U[a:b], x)

    with cf.ThreadPoolExecutor(THREADS) as ex:
        list(ex.map(job, range(THREADS)))
    return out


def pack(V: np.ndarray) -> np.ndarray:
    """oracle.pack on row chunks in threads."""
    n = V.shape[0]
    if n < 4096:
        return oracle.pack(V)
    bounds = np.linspace(0, n, THREADS + 1).astype(np.int64)
    parts = [None] * THREADS

    def job(i):
        parts[i] = oracle.pack(V[bounds[i]:bounds[i + 1]])

    with cf.ThreadPoolExecutor(THREADS) as ex:
        list(ex.map(job, range(THREADS)))
    return np.concatenate(parts)


def knn(Vq: np.ndarray, Vs: np.ndarray, k: int):
    nq = Vq.shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    dist = np.empty((nq, k), dtype=np.int32)

    def job(q):
        ids[q:q + 1], dist[q:q + 1] = oracle.knn(Vq[q:q + 1], Vs, k)

    with cf.ThreadPoolExecutor(min(THREADS, nq)) as ex:
        list(ex.map(job, range(nq)))
    return ids, dist


def knn_i8q(Q8: np.ndarray, Vs: np.ndarray, k: int):
    nq = Q8.shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    score = np.empty((nq, k), dtype=np.int32)

    def job(q):
        ids[q:q + 1], score[q:q + 1] = oracle.knn_i8q(Q8[q:q + 1], Vs, k)

    with cf.ThreadPoolExecutor(min(THREADS, nq)) as ex:
        list(ex.map(job, range(nq)))
    return ids, score


def check_knn_sampled(Vq_row, ids_row, dist_row, V_returned, V_sample, sample_idx):
    """Properties that hold at any size, checked by the oracle one row at a time:
    the returned distances are the oracle's Delta of the returned rows, the
    list is strictly increasing in (Delta, id), and no sampled row that was
    left out beats the k-th returned (Delta, id)."""
    k = len(ids_row)
    assert len(set(ids_row.tolist())) == k
    for j in range(k):
        assert oracle.delta(Vq_row, V_returned[j]) == dist_row[j], (j, ids_row[j])
    keys = list(zip(dist_row.tolist(), ids_row.tolist()))
    assert all(keys[j] < keys[j + 1] for j in range(k - 1))
    si, sd = oracle.knn(Vq_row[None], V_sample, len(sample_idx))
    kth = keys[-1]
    chosen = set(ids_row.tolist())
    for local, dd in zip(si[0], sd[0]):
        g = int(sample_idx[local])
        if (int(dd), g) < kth:
            assert g in chosen, (g, int(dd), kth)
        else:
            break
