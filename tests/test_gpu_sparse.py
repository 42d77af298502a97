"""Sparse small-x codes (Sec. 6, "different EVPs") and the masked-addition
scan over them: the packed-to-sparse conversion is bit-exact against the
oracle's sparse form, and the scan returns the oracle's exhaustive kNN (ids
and Delta) -- the same results as the bitplane scan -- over ragged sizes,
several passes of 4 queries, k up to the path's limit, and at the full
10M x 768 (x = 64) size."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth
from oracle_par import encode as par_encode, knn as par_knn

pytestmark = pytest.mark.gpu


def _sparse_host(E):
    return E.cpu().numpy().view(np.uint16)


@pytest.mark.parametrize("d,x", [(384, 8), (768, 64), (1000, 120), (128, 120)])
def test_pack_sparse_matches_oracle(evp_lib, dev, d, x):
    U = synth.mixture_numpy(3000, d, n_centres=16, anisotropic=True, stream=900 + d)
    st = evp_lib.new_status(dev)
    T = evp_lib.encode(torch.from_numpy(U).to(dev), x, status=st)
    E = evp_lib.pack_sparse(T, d, x, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    np.testing.assert_array_equal(_sparse_host(E), oracle.sparse_pack(oracle.encode(U, x), x))


def test_pack_sparse_flags_wrong_counts(evp_lib, dev):
    d, x = 256, 16
    V = synth.ternary_random(40, d, x, stream=901)
    V[7, :] = 0
    V[7, :10] = 1                                  # 10 non-zeros instead of 16
    T = torch.from_numpy(oracle.pack(V).view(np.int64)).to(dev)
    st = evp_lib.new_status(dev)
    E = evp_lib.pack_sparse(T, d, x, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == evp_lib.EVP_ERR_RANGE
    ok = [i for i in range(40) if i != 7]
    np.testing.assert_array_equal(_sparse_host(E)[ok], oracle.sparse_pack(V[ok], x))


@pytest.mark.parametrize("ns,d,x,nq,k", [
    (20_011, 768, 64, 1, 10),
    (20_011, 768, 64, 5, 100),       # two passes (4 + 1), ragged tail
    (9_000, 384, 120, 13, 256),      # four passes, the path's largest k
    (5_000, 1000, 8, 4, 1),
    (300, 128, 16, 3, 256),          # k close to ns
])
def test_sparse_scan_matches_oracle(evp_lib, dev, ns, d, x, nq, k):
    U = synth.mixture_numpy(ns, d, n_centres=32, anisotropic=True, stream=910 + d)
    Qf = synth.mixture_numpy(nq, d, n_centres=32, anisotropic=True, stream=911 + d)
    st = evp_lib.new_status(dev)
    S = evp_lib.encode(torch.from_numpy(U).to(dev), x, status=st)
    Q = evp_lib.encode(torch.from_numpy(Qf).to(dev), x, status=st)
    E = evp_lib.pack_sparse(S, d, x, status=st)
    ids, dist = evp_lib.ternary_knn_sparse(Q, E, d, x, k, status=st)
    ids_b, dist_b = evp_lib.ternary_knn(Q, S, d, x, k, status=st, path=evp_lib.PATH_POPC)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    oi, od = par_knn(oracle.encode(Qf, x), par_encode(U, x), k)
    np.testing.assert_array_equal(ids.cpu().numpy(), oi)
    np.testing.assert_array_equal(dist.cpu().numpy(), od)
    assert torch.equal(ids, ids_b) and torch.equal(dist, dist_b)


def test_sparse_limits(evp_lib, dev):
    lib = evp_lib.load()
    assert lib.ternary_knn_sparse_workspace(4, 1000, 768, 4, 10) == 0     # x < 8
    assert lib.ternary_knn_sparse_workspace(4, 1000, 768, 100, 10) == 0   # x not a multiple of 8
    assert lib.ternary_knn_sparse_workspace(4, 1000, 768, 128, 10) == 0   # x > 120
    assert lib.ternary_knn_sparse_workspace(4, 1000, 768, 64, 300) == 0   # k > 256
    assert lib.ternary_knn_sparse_workspace(4, 1000, 768, 64, 100) > 0


def test_sparse_10m_exhaustive(evp_lib, dev):
    """10M x 768 at x = 64 (the paper's small-x case at d = 768), 8 queries
    (two passes): the oracle's exhaustive kNN over all rows."""
    n, d, x, nq, k = 10_000_000, 768, 64, 8, 100
    U = synth.mixture_torch(n, d, n_centres=1024, anisotropic=True, stream=synth.STREAM_DB,
                            device=dev)
    Q = synth.mixture_torch(nq, d, n_centres=1024, anisotropic=True,
                            stream=synth.STREAM_QUERIES, device=dev)
    st = evp_lib.new_status(dev)
    S = evp_lib.encode(U, x, status=st)
    Tq = evp_lib.encode(Q, x, status=st)
    E = evp_lib.pack_sparse(S, d, x, status=st)
    ids, dist = evp_lib.ternary_knn_sparse(Tq, E, d, x, k, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    sel = [0, 3, 4, 7]
    Vs = par_encode(U.cpu().numpy(), x)
    oi, od = par_knn(oracle.encode(Q.cpu().numpy()[sel], x), Vs, k)
    np.testing.assert_array_equal(ids.cpu().numpy()[sel], oi)
    np.testing.assert_array_equal(dist.cpu().numpy()[sel], od)
