"""The asymmetric scan (single-operand translation, Sec. 6): int8 queries
against the ternary database with the masked-addition score of Sec. 5.1.2,
on the tensor cores.  Quantisation and search results are compared with the
oracle bit for bit (ids and scores), over ragged sizes, several passes of 32
queries, k up to the path's limit, ties and degenerate queries, and at the
full 10M x 768 size against the oracle's exhaustive search."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth
from oracle_par import encode as par_encode, knn_i8q as par_knn_i8q

pytestmark = pytest.mark.gpu


def test_quantize_matches_oracle(evp_lib, dev):
    Q = synth.mixture_numpy(300, 384, n_centres=16, stream=801)
    Q[3] = 0.0                                            # zero row -> zeros
    Q[4, :] = 0.0
    Q[4, 7] = -2.5e-3                                     # one non-zero -> -127
    Q[5, :10] = np.float32([127.0, 2.5, 3.5, -2.5, -3.5, 0.5, -0.5, 1.5, 126.5, 0.0])
    Q[5, 10:] = 0.0
    st = evp_lib.new_status(dev)
    q8 = evp_lib.quantize_i8(torch.from_numpy(Q).to(dev), status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    np.testing.assert_array_equal(q8.cpu().numpy(), oracle.quantize_i8(Q))
    Q[9, 100] = np.nan
    st = evp_lib.new_status(dev)
    evp_lib.quantize_i8(torch.from_numpy(Q).to(dev), status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == evp_lib.EVP_ERR_NONFINITE


@pytest.mark.parametrize("ns,d,x,nq,k", [
    (20_000, 384, 128, 1, 10),
    (20_000, 384, 128, 16, 100),
    (20_011, 384, 256, 33, 50),      # ragged tail, two passes (32 + 1)
    (9_999, 768, 512, 70, 256),      # three passes, the path's largest k
    (5_000, 128, 40, 17, 1),
    (3_000, 768, 64, 32, 200),
])
def test_i8q_matches_oracle(evp_lib, dev, ns, d, x, nq, k):
    U = synth.mixture_numpy(ns, d, n_centres=32, anisotropic=True, stream=810 + d)
    Qf = synth.mixture_numpy(nq, d, n_centres=32, anisotropic=True, stream=811 + d)
    st = evp_lib.new_status(dev)
    S = evp_lib.encode(torch.from_numpy(U).to(dev), x, status=st)
    q8 = evp_lib.quantize_i8(torch.from_numpy(Qf).to(dev), status=st)
    ids, sc = evp_lib.ternary_knn_i8q(q8, S, d, x, k, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    oi, osc = par_knn_i8q(oracle.quantize_i8(Qf), par_encode(U, x), k)
    np.testing.assert_array_equal(ids.cpu().numpy(), oi)
    np.testing.assert_array_equal(sc.cpu().numpy(), osc)


def test_i8q_ties_and_degenerate_queries(evp_lib, dev):
    d, x, ns, k = 384, 128, 12_000, 40
    U = synth.mixture_numpy(ns, d, n_centres=8, stream=820)
    U[5000:5100] = U[17]                     # 101 identical rows: exact score ties
    st = evp_lib.new_status(dev)
    S = evp_lib.encode(torch.from_numpy(U).to(dev), x, status=st)
    q8 = np.zeros((4, d), dtype=np.int8)     # all-zero query: every score 0, ids 0..k-1
    q8[1, 3] = 127                           # one non-zero element
    q8[2] = oracle.quantize_i8(U[17:18])[0]  # the duplicated row itself
    q8[3] = -q8[2]
    ids, sc = evp_lib.ternary_knn_i8q(torch.from_numpy(q8).to(dev), S, d, x, k, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    oi, osc = oracle.knn_i8q(q8, oracle.encode(U, x), k)
    np.testing.assert_array_equal(ids.cpu().numpy(), oi)
    np.testing.assert_array_equal(sc.cpu().numpy(), osc)
    assert ids.cpu().numpy()[0].tolist() == list(range(k))


def test_i8q_limits(evp_lib, dev):
    assert evp_lib.load().ternary_knn_i8q_workspace(4, 1000, 1024, 10) == 0   # d > 768
    assert evp_lib.load().ternary_knn_i8q_workspace(4, 1000, 384, 300) == 0   # k > 256
    S = torch.zeros((1000, 2 * evp_lib.words(1024)), dtype=torch.int64, device=dev)
    q8 = torch.zeros((4, 1024), dtype=torch.int8, device=dev)
    with pytest.raises(evp_lib.EvpError) as e:
        evp_lib.ternary_knn_i8q(q8, S, 1024, 256, 10)
    assert e.value.code == evp_lib.EVP_ERR_UNSUPPORTED


def test_i8q_10m_exhaustive(evp_lib, dev):
    """10M x 768, x = 512, 32 queries (one pass): the oracle's exhaustive
    masked-addition search over all 10M rows, on queries of both halves of
    the pass (the two epilogue warp groups)."""
    n, d, x, nq, k = 10_000_000, 768, 512, 32, 100
    U = synth.mixture_torch(n, d, n_centres=1024, anisotropic=True, stream=synth.STREAM_DB,
                            device=dev)
    Q = synth.mixture_torch(nq, d, n_centres=1024, anisotropic=True,
                            stream=synth.STREAM_QUERIES, device=dev)
    st = evp_lib.new_status(dev)
    S = evp_lib.encode(U, x, status=st)
    q8 = evp_lib.quantize_i8(Q, status=st)
    ids, sc = evp_lib.ternary_knn_i8q(q8, S, d, x, k, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    sel = [0, 15, 16, 31]
    Vs = par_encode(U.cpu().numpy(), x)
    oi, osc = par_knn_i8q(oracle.quantize_i8(Q.cpu().numpy()[sel]), Vs, k)
    np.testing.assert_array_equal(ids.cpu().numpy()[sel], oi)
    np.testing.assert_array_equal(sc.cpu().numpy()[sel], osc)
