"""The tensor-core scan with capped lists (kl < k keys per query and slice:
the smallest power of two >= 16 with kl x slices >= 4k, at most 128) against
the oracle, including databases
ordered so that a query's k nearest rows are contiguous -- they then fall
into one or two slices, far more than a capped list keeps, and only the
repair pass (a rescan of those slices) can make the result exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth

pytestmark = pytest.mark.gpu

PATH_MMA = 2


def _knn(evp, Vq, Vs, d, x, k, dev):
    Qd = torch.from_numpy(oracle.pack(Vq).view(np.int64)).to(dev)
    Sd = torch.from_numpy(oracle.pack(Vs).view(np.int64)).to(dev)
    st = evp.new_status(dev)
    ids, dist = evp.ternary_knn(Qd, Sd, d, x, k, status=st, path=PATH_MMA)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return ids.cpu().numpy(), dist.cpu().numpy()


@pytest.mark.parametrize("nq,k", [(8, 700), (200, 300), (3, 1024), (200, 100), (40, 33)])
def test_contiguous_neighbours_are_repaired(evp_lib, dev, nq, k):
    d, x, ns = 384, 128, 20_000
    U = synth.mixture_numpy(ns, d, n_centres=32, stream=900)
    Qf = synth.mixture_numpy(nq, d, n_centres=32, stream=901)
    Vs, Vq = oracle.encode(U, x), oracle.encode(Qf, x)
    # query 0's rows nearest first: its k nearest occupy the first k rows
    order, _ = oracle.knn(Vq[:1], Vs, ns)
    Vs = Vs[order[0]]
    ids, dist = _knn(evp_lib, Vq, Vs, d, x, k, dev)
    oi, od = oracle.knn(Vq, Vs, k)
    np.testing.assert_array_equal(dist, od)
    np.testing.assert_array_equal(ids, oi)
    assert np.array_equal(np.sort(ids[0]), np.arange(k))   # the contiguous block itself


@pytest.mark.parametrize("k", [33, 100, 129, 500, 1000])
def test_random_order_large_k(evp_lib, dev, k):
    d, x, ns, nq = 256, 171, 60_000, 100
    U = synth.mixture_numpy(ns, d, n_centres=64, stream=910)
    Qf = synth.mixture_numpy(nq, d, n_centres=64, stream=911)
    Vs, Vq = oracle.encode(U, x), oracle.encode(Qf, x)
    ids, dist = _knn(evp_lib, Vq, Vs, d, x, k, dev)
    oi, od = oracle.knn(Vq, Vs, k)
    np.testing.assert_array_equal(dist, od)
    np.testing.assert_array_equal(ids, oi)
