"""Parity at the full workload sizes.

* 1,000,000 x 768 Gaussian mixture (1,024 centres, anisotropic scales),
  x in {64, 256, 384}, k = 100: the oracle encodes the whole database and
  checks several queries exhaustively (bit-exact ids and Delta).
* 10,000,000 x 768, x = 512, 1,024 queries, shortlist 100 then rerank to
  10 -- the benchmark's launch configuration -- checked on sampled queries
  through properties the oracle computes row by row.
* 10,000,000 x 1024, x = 256, 4,096 queries (the large dense contraction):
  the resident database's tensor-core scan, shortlist 100, rerank to 10,
  checked the same way.
* 10,000,000 x 768, 16 queries on the packed tensor-core scan: identical to
  the popcount scan and checked the same way on sampled rows.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth
from oracle_par import check_knn_sampled, encode as par_encode, knn as par_knn
from test_gpu_rerank import check_rerank

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def db_1m(dev):
    U = synth.mixture_torch(1_000_000, 768, n_centres=1024, anisotropic=True,
                            stream=synth.STREAM_DB, device=dev)
    Q = synth.mixture_torch(40, 768, n_centres=1024, anisotropic=True,
                            stream=synth.STREAM_QUERIES, device=dev)
    return U, Q, U.cpu().numpy(), Q.cpu().numpy()


@pytest.mark.parametrize("x,path", [(64, 1), (256, 1), (384, 1), (256, 2), (64, 2),
                                    (64, 3), (256, 3), (384, 3)])
def test_scale_1m_exhaustive_queries(evp_lib, dev, db_1m, x, path):
    U, Q, U_h, Q_h = db_1m
    d, k = 768, 100
    st = evp_lib.new_status(dev)
    Ts = evp_lib.encode(U, x, status=st)
    Tq = evp_lib.encode(Q, x, status=st)
    ids, dist = evp_lib.ternary_knn(Tq, Ts, d, x, k, status=st, path=path)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Vs = par_encode(U_h, x)
    Vq = oracle.encode(Q_h, x)
    # encode: bit-exact on the full database
    np.testing.assert_array_equal(Ts.cpu().numpy().view(np.uint64), oracle.pack(Vs))
    sel = [0, 15, 16, 39]   # first pass, its last query, second pass, last pass
    oi, od = par_knn(Vq[sel], Vs, k)
    np.testing.assert_array_equal(ids.cpu().numpy()[sel], oi)
    np.testing.assert_array_equal(dist.cpu().numpy()[sel], od)


def test_bench_workload_10m_sampled(evp_lib, dev):
    n, d, x, nq, n_sl, k = 10_000_000, 768, 512, 1024, 100, 10
    U = synth.mixture_torch(n, d, n_centres=1024, anisotropic=True, stream=synth.STREAM_DB,
                            device=dev)
    Q = synth.mixture_torch(nq, d, n_centres=1024, anisotropic=True,
                            stream=synth.STREAM_QUERIES, device=dev)
    st = evp_lib.new_status(dev)
    Ts = evp_lib.encode(U, x, status=st)
    Tq = evp_lib.encode(Q, x, status=st)
    sl, sd = evp_lib.ternary_knn(Tq, Ts, d, x, n_sl, status=st)
    rid, rsc = evp_lib.rerank(Q, U, sl, k, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    rng = np.random.default_rng(123)
    sample_idx = np.sort(rng.choice(n, 50_000, replace=False))
    U_sample = U[torch.from_numpy(sample_idx).to(dev)].cpu().numpy()
    V_sample = par_encode(U_sample, x)
    # encode bit-exact on the sampled rows
    np.testing.assert_array_equal(Ts[torch.from_numpy(sample_idx).to(dev)].cpu().numpy()
                                  .view(np.uint64), oracle.pack(V_sample))
    Q_h = Q.cpu().numpy()
    Vq = oracle.encode(Q_h, x)
    sl_h, sd_h = sl.cpu().numpy(), sd.cpu().numpy()
    for q in (0, 17, 511, 1023):
        rows = U[torch.from_numpy(sl_h[q]).to(dev)].cpu().numpy()
        check_knn_sampled(Vq[q], sl_h[q], sd_h[q], oracle.encode(rows, x), V_sample, sample_idx)
        # rerank of that query's shortlist against float64
        S_rows = rows
        local = np.arange(n_sl, dtype=np.int64)[None, :]
        gi = rid.cpu().numpy()[q:q + 1]
        g_local = np.array([[int(np.where(sl_h[q] == i)[0][0]) for i in gi[0]]])
        check_rerank(g_local, rsc.cpu().numpy()[q:q + 1], Q_h[q:q + 1], S_rows, local, k)


def test_dense_contraction_10m_1024_sampled(evp_lib, dev):
    n, d, x, nq, n_sl, k = 10_000_000, 1024, 256, 4096, 100, 10
    U = synth.mixture_torch(n, d, n_centres=1024, anisotropic=True, stream=synth.STREAM_DB,
                            device=dev)
    Q = synth.mixture_torch(nq, d, n_centres=1024, anisotropic=True,
                            stream=synth.STREAM_QUERIES, device=dev)
    st = evp_lib.new_status(dev)
    Ts = evp_lib.encode(U, x, status=st)
    Tq = evp_lib.encode(Q, x, status=st)
    db = evp_lib.Database(Ts, U, d, x)
    sl, sd = db.knn(Tq, n_sl, status=st)
    rid, rsc = db.search(Q, n_sl, k, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    rng = np.random.default_rng(321)
    sample_idx = np.sort(rng.choice(n, 30_000, replace=False))
    U_sample = U[torch.from_numpy(sample_idx).to(dev)].cpu().numpy()
    V_sample = par_encode(U_sample, x)
    np.testing.assert_array_equal(Ts[torch.from_numpy(sample_idx).to(dev)].cpu().numpy()
                                  .view(np.uint64), oracle.pack(V_sample))
    Q_h = Q.cpu().numpy()
    sel = (0, 129, 2048, 4095)   # several query tiles and both CTAs of a pair
    Vq = oracle.encode(Q_h[list(sel)], x)
    sl_h, sd_h = sl.cpu().numpy(), sd.cpu().numpy()
    rid_h, rsc_h = rid.cpu().numpy(), rsc.cpu().numpy()
    for i, q in enumerate(sel):
        rows = U[torch.from_numpy(sl_h[q]).to(dev)].cpu().numpy()
        check_knn_sampled(Vq[i], sl_h[q], sd_h[q], oracle.encode(rows, x), V_sample, sample_idx)
        # the search's rerank reorders this same shortlist
        gi = rid_h[q]
        g_local = np.array([[int(np.where(sl_h[q] == j)[0][0]) for j in gi]])
        local = np.arange(n_sl, dtype=np.int64)[None, :]
        check_rerank(g_local, rsc_h[q:q + 1], Q_h[q:q + 1], rows, local, k)
    db.close()


def test_packed_path_10m_16_queries_sampled(evp_lib, dev):
    """The packed tensor-core scan at the full 10M x 768 size with 16
    queries (the launch `bench.py --batch 16` times): results identical to
    the popcount scan's, and checked against the oracle on sampled rows."""
    n, d, x, nq, k = 10_000_000, 768, 512, 16, 100
    U = synth.mixture_torch(n, d, n_centres=1024, anisotropic=True, stream=synth.STREAM_DB,
                            device=dev)
    Q = synth.mixture_torch(nq, d, n_centres=1024, anisotropic=True,
                            stream=synth.STREAM_QUERIES, device=dev)
    st = evp_lib.new_status(dev)
    Ts = evp_lib.encode(U, x, status=st)
    Tq = evp_lib.encode(Q, x, status=st)
    db = evp_lib.Database(Ts, None, d, x, tensor_copy=False)
    ids, dist = db.knn(Tq, k, status=st, path=3)
    ids_a, dist_a = db.knn(Tq, k, status=st)          # the automatic choice (packed here)
    ids_p, dist_p = db.knn(Tq, k, status=st, path=1)  # the popcount scan
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert torch.equal(ids, ids_p) and torch.equal(dist, dist_p)
    assert torch.equal(ids, ids_a) and torch.equal(dist, dist_a)
    rng = np.random.default_rng(654)
    sample_idx = np.sort(rng.choice(n, 40_000, replace=False))
    U_sample = U[torch.from_numpy(sample_idx).to(dev)].cpu().numpy()
    V_sample = par_encode(U_sample, x)
    Q_h = Q.cpu().numpy()
    sel = (0, 7, 15)
    Vq = oracle.encode(Q_h[list(sel)], x)
    ids_h, dist_h = ids.cpu().numpy(), dist.cpu().numpy()
    for i, q in enumerate(sel):
        rows = U[torch.from_numpy(ids_h[q]).to(dev)].cpu().numpy()
        check_knn_sampled(Vq[i], ids_h[q], dist_h[q], oracle.encode(rows, x), V_sample, sample_idx)
    db.close()
