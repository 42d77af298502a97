"""Resident database handle (evp_db_*): identical results to the stateless
calls, and the whole float-query path against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth
from test_gpu_rerank import check_rerank

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_db(dev, evp_lib):
    d, x = 384, 128
    U = synth.mixture_numpy(10_000, d, n_centres=64, stream=synth.STREAM_DB)
    Qf = synth.mixture_numpy(100, d, n_centres=64, stream=synth.STREAM_QUERIES)
    Ud = torch.from_numpy(U).to(dev)
    T = evp_lib.encode(Ud, x)
    return d, x, U, Qf, Ud, T


@pytest.mark.parametrize("tensor_copy", [True, False])
@pytest.mark.parametrize("path", [0, 1, 2, 3])
def test_db_knn_matches_oracle(evp_lib, dev, small_db, tensor_copy, path):
    d, x, U, Qf, Ud, T = small_db
    db = evp_lib.Database(T, Ud, d, x, tensor_copy=tensor_copy)
    Tq = evp_lib.encode(torch.from_numpy(Qf).to(dev), x)
    st = evp_lib.new_status(dev)
    ids, dist = db.knn(Tq, 10, status=st, path=path)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    oi, od = oracle.knn(oracle.encode(Qf, x), oracle.encode(U, x), 10)
    np.testing.assert_array_equal(ids.cpu().numpy(), oi)
    np.testing.assert_array_equal(dist.cpu().numpy(), od)
    db.close()


@pytest.mark.parametrize("nq,n_sl,k", [(100, 100, 10), (7, 50, 5), (40, 300, 30), (1, 1, 1)])
def test_db_search_whole_path(evp_lib, dev, small_db, nq, n_sl, k):
    d, x, U, Qf, Ud, T = small_db
    db = evp_lib.Database(T, Ud, d, x)
    Q = torch.from_numpy(Qf[:nq]).to(dev)
    st = evp_lib.new_status(dev)
    ids, scores = db.search(Q, n_sl, k, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    # oracle: encode, exhaustive shortlist by Delta, float64 rerank
    oi, _ = oracle.knn(oracle.encode(Qf[:nq], x), oracle.encode(U, x), n_sl)
    check_rerank(ids.cpu().numpy(), scores.cpu().numpy(), Qf[:nq], U, oi, k)
    # host-buffer form gives the same bytes
    ids_h = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    sc_h = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    db.search_host(torch.from_numpy(Qf[:nq].copy()).pin_memory(), n_sl, k, ids_h, sc_h, status=st)
    torch.cuda.synchronize()
    assert torch.equal(ids_h, ids.cpu()) and torch.equal(sc_h, scores.cpu())
    db.close()


def test_db_argument_errors(evp_lib, dev, small_db):
    d, x, U, Qf, Ud, T = small_db
    db = evp_lib.Database(T, None, d, x, tensor_copy=False)
    Q = torch.from_numpy(Qf[:4]).to(dev)
    with pytest.raises(evp_lib.EvpError):
        db.search(Q, 10, 5)            # no float rows to rerank against
    db.close()
    db = evp_lib.Database(T, Ud, d, x)
    with pytest.raises(evp_lib.EvpError):
        db.search(Q, 5, 10)            # shortlist shorter than k
    with pytest.raises(evp_lib.EvpError):
        evp_lib.Database(T, Ud, d, d + 1)
    db.close()
