"""evp_merge_topk: a database split into P row shards, each searched on its
own, merges into exactly the unsharded ternary_knn result."""
import numpy as np
import pytest
import torch

from paper_2506_00528_gb300 import dist as evp_dist
from paper_2506_00528_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("P,k", [(2, 10), (3, 100), (8, 50), (5, 1024)])
def test_sharded_search_equals_whole(evp_lib, dev, P, k):
    d, x, ns = 384, 128, 40_000
    U = torch.from_numpy(synth.mixture_numpy(ns, d, n_centres=32, stream=70)).to(dev)
    Q = torch.from_numpy(synth.mixture_numpy(37, d, n_centres=32, stream=71)).to(dev)
    S, Tq = evp_lib.encode(U, x), evp_lib.encode(Q, x)
    whole_i, whole_d = evp_lib.ternary_knn(Tq, S, d, x, k)
    ids, dd = [], []
    for r in range(P):
        r0, r1 = evp_dist.shard_bounds(ns, P, r)
        kk = min(k, r1 - r0)
        i, dist_ = evp_lib.ternary_knn(Tq, S[r0:r1].contiguous(), d, x, kk)
        pad_i = torch.full((37, k), -1, dtype=torch.int64, device=dev)
        pad_d = torch.full((37, k), -1, dtype=torch.int32, device=dev)
        pad_i[:, :kk] = i + r0
        pad_d[:, :kk] = dist_
        ids.append(pad_i)
        dd.append(pad_d)
    mi, md = evp_lib.merge_topk(torch.stack(ids).contiguous(), torch.stack(dd).contiguous(), k)
    torch.cuda.synchronize()
    assert torch.equal(mi, whole_i) and torch.equal(md, whole_d)
