"""Multi-process host logic on CPU (gloo, world size 2): row-shard bounds,
the all-gather of per-shard (Delta, id) lists and their merge, and the
max-over-ranks / sum-over-ranks aggregation.  The oracle plays the part of
each rank's scan and of the merge."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2506_00528_gb300 import dist as evp_dist
from paper_2506_00528_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_merge(ids, dd, k):
    P, nq, _ = ids.shape
    out_i = np.full((nq, k), -1, dtype=np.int64)
    out_d = np.full((nq, k), -1, dtype=np.int32)
    for q in range(nq):
        keys = [(int(dd[p, q, j]), int(ids[p, q, j])) for p in range(P) for j in range(ids.shape[2])
                if ids[p, q, j] >= 0]
        keys.sort()
        for j, (d_, i_) in enumerate(keys[:k]):
            out_i[q, j], out_d[q, j] = i_, d_
    return torch.from_numpy(out_i), torch.from_numpy(out_d)


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d, x, ns, k = 64, 43, 3001, 25
    U = synth.mixture_numpy(ns, d, n_centres=16, stream=61)
    Qf = synth.mixture_numpy(9, d, n_centres=16, stream=62)
    r0, r1 = evp_dist.shard_bounds(ns, world, rank)
    Vs = oracle.encode(U[r0:r1], x)
    Vq = oracle.encode(Qf, x)
    ids, dd = oracle.knn(Vq, Vs, k)
    gi, gd = evp_dist.gather_and_merge(torch.from_numpy(ids), torch.from_numpy(dd), k,
                                       lambda a, b, kk: _oracle_merge(a.numpy(), b.numpy(), kk),
                                       row_offset=r0)
    units, ms = evp_dist.aggregate(10 * (rank + 1), 5.0 + rank)
    if rank == 0:
        np.savez(out_path, ids=gi.numpy(), dist=gd.numpy(), units=units, ms=ms)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_row_shards_merge_to_unsharded_result(tmp_path, world):
    out = str(tmp_path / "res.npz")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    res = np.load(out)
    d, x, ns, k = 64, 43, 3001, 25
    U = synth.mixture_numpy(ns, d, n_centres=16, stream=61)
    Qf = synth.mixture_numpy(9, d, n_centres=16, stream=62)
    oi, od = oracle.knn(oracle.encode(Qf, x), oracle.encode(U, x), k)
    np.testing.assert_array_equal(res["ids"], oi)
    np.testing.assert_array_equal(res["dist"], od)
    assert float(res["units"]) == 30.0 and float(res["ms"]) == 6.0


def test_shard_bounds_cover_rows():
    for ns in (1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            bounds = [evp_dist.shard_bounds(ns, world, r) for r in range(world)]
            assert bounds[0][0] == 0 and bounds[-1][1] == ns
            assert all(b[1] == n[0] for b, n in zip(bounds, bounds[1:]))
            sizes = [b[1] - b[0] for b in bounds]
            assert max(sizes) - min(sizes) <= 1
