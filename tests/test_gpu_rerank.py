"""rerank on the GPU against the float64 oracle.

Tolerance (a reading of the precision the method needs): every float32
score within 1e-5 * sum_i |q_i s_i| of the float64 score; the returned ids
must be a valid top-k -- any difference from the oracle's list only among
entries whose float64 scores lie within twice that tolerance.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth

pytestmark = pytest.mark.gpu
REL = 1e-5


def check_rerank(gi, gs, Q, S, sl, k):
    nq, n = sl.shape
    oi, os_, oa = oracle.rerank(Q, S, sl, n)          # every entry, sorted
    for q in range(nq):
        valid = int((oi[q] >= 0).sum())
        score = {int(i): (float(s), float(a)) for i, s, a in zip(oi[q], os_[q], oa[q]) if i >= 0}
        kk = min(k, valid)
        assert np.all(gi[q, kk:] == -1) and np.all(np.isneginf(gs[q, kk:]))
        ids = [int(v) for v in gi[q, :kk]]
        assert len(set(ids)) == kk and all(i in score for i in ids)
        tol = [REL * score[i][1] for i in ids]
        for j, i in enumerate(ids):
            assert abs(gs[q, j] - score[i][0]) <= tol[j], (q, j, gs[q, j], score[i])
        # GPU order is by its own scores, descending, ties by id
        for j in range(kk - 1):
            assert (gs[q, j] > gs[q, j + 1]) or (gs[q, j] == gs[q, j + 1] and ids[j] < ids[j + 1])
        # valid top-k against float64: anything left out is not clearly better
        kth = score[ids[-1]][0] if kk else 0.0
        chosen = set(ids)
        for i, (s64, a) in score.items():
            if i not in chosen:
                assert s64 <= kth + 2 * REL * max(a, score[ids[-1]][1]), (q, i, s64, kth)


@pytest.mark.parametrize("d,n,k", [(384, 100, 10), (768, 1000, 100), (1024, 100, 10),
                                   (100, 37, 37), (3, 5, 2), (1001, 64, 1), (4096, 16, 8),
                                   (768, 4096, 1000)])
def test_rerank_matches_float64(evp_lib, dev, d, n, k):
    ns, nq = 5000, 9
    S = synth.mixture_numpy(ns, d, n_centres=8, anisotropic=True, stream=700 + d)
    Q = synth.mixture_numpy(nq, d, n_centres=8, anisotropic=True, stream=800 + d)
    rng = np.random.default_rng(d + n)
    sl = np.stack([rng.choice(ns, n, replace=False) for _ in range(nq)]).astype(np.int64)
    st = evp_lib.new_status(dev)
    gi, gs = evp_lib.rerank(torch.from_numpy(Q).to(dev), torch.from_numpy(S).to(dev),
                            torch.from_numpy(sl).to(dev), k, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check_rerank(gi.cpu().numpy(), gs.cpu().numpy(), Q, S, sl, k)


def test_rerank_empty_entries_ties_and_range(evp_lib, dev):
    S = np.array([[1, 0, 0, 0], [0.5, 0.5, 0, 0], [0, 1, 0, 0],
                  [0.5, 0.5, 0, 0], [-1, 0, 0, 0]], dtype=np.float32)
    Q = np.array([[1, 0, 0, 0], [0, 0, 0, 1]], dtype=np.float32)
    sl = np.array([[4, 3, 1, 0, -1, 2], [0, 1, 2, 3, 4, -1]], dtype=np.int64)
    st = evp_lib.new_status(dev)
    gi, gs = evp_lib.rerank(torch.from_numpy(Q).to(dev), torch.from_numpy(S).to(dev),
                            torch.from_numpy(sl).to(dev), 5, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    oi, os_, _ = oracle.rerank(Q, S, sl, 5)
    np.testing.assert_array_equal(gi.cpu().numpy(), oi)
    np.testing.assert_array_equal(gs.cpu().numpy(), os_.astype(np.float32))
    # an id outside [-1, ns) is reported and skipped
    bad = torch.tensor([[0, 9, 2]], dtype=torch.int64, device=dev)
    st = evp_lib.new_status(dev)
    gi, _ = evp_lib.rerank(torch.from_numpy(Q[:1]).to(dev), torch.from_numpy(S).to(dev), bad, 3,
                           status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == evp_lib.EVP_ERR_RANGE
    assert gi.cpu().numpy()[0].tolist() == [0, 2, -1]


def test_rerank_nonfinite(evp_lib, dev):
    S = synth.mixture_numpy(50, 32, stream=9)
    S[3, 5] = np.nan
    Q = synth.mixture_numpy(2, 32, stream=10)
    sl = torch.arange(50, device=dev).repeat(2, 1)
    st = evp_lib.new_status(dev)
    evp_lib.rerank(torch.from_numpy(Q).to(dev), torch.from_numpy(S).to(dev), sl, 5, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == evp_lib.EVP_ERR_NONFINITE
