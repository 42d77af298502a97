"""Parity at the full workload sizes.

* 1,000,000 x 768 Gaussian mixture (1,024 centres, anisotropic scales),
  x in {64, 256, 384}, k = 100: the oracle encodes the whole database and
  checks several queries exhaustively (bit-exact ids and Delta).
* 10,000,000 x 768, x = 512 (the benchmark's database): every code of the
  database compared with the oracle's, and the exhaustive kNN (Sec. 5.3)
  of the oracle over all 10M rows compared id by id and Delta by Delta with
  each scan path -- the popcount scan (40 queries, three passes), the fp4
  tensor-core scan in the benchmark's launch configuration (1,024 queries,
  shortlist 100, then the rerank to 10) and the packed tensor-core scan
  (16 and 64 queries) -- on queries spread over passes, query tiles and
  both CTAs of a pair.
* 10,000,000 x 1024, x = 256 (the large dense contraction): every code
  compared, and the resident database's tensor-core scan of 4,096 queries
  plus the popcount scan compared exhaustively on sampled queries; the
  4,096-query batch is also checked through the sampled-row properties.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth
from oracle_par import check_knn_sampled, encode as par_encode, knn as par_knn
from oracle_par import pack as par_pack
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


def _host_codes(T):
    return T.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module")
def db_10m_768(dev):
    """The benchmark's database: 10M x 768, x = 512, encoded on the GPU and,
    row for row, by the oracle."""
    n, d, x = 10_000_000, 768, 512
    U = synth.mixture_torch(n, d, n_centres=1024, anisotropic=True, stream=synth.STREAM_DB,
                            device=dev)
    Q = synth.mixture_torch(1024, d, n_centres=1024, anisotropic=True,
                            stream=synth.STREAM_QUERIES, device=dev)
    import paper_2506_00528_gb300.evp as evp
    evp.load()
    st = evp.new_status(dev)
    Ts = evp.encode(U, x, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    U_h = U.cpu().numpy()
    Vs = par_encode(U_h, x)
    del U_h
    Q_h = Q.cpu().numpy()
    return {"n": n, "d": d, "x": x, "U": U, "Q": Q, "Q_h": Q_h, "Ts": Ts, "Vs": Vs,
            "Vq": oracle.encode(Q_h, x)}


def test_10m_768_encode_every_row(evp_lib, db_10m_768):
    D = db_10m_768
    np.testing.assert_array_equal(_host_codes(D["Ts"]), par_pack(D["Vs"]))


def _check_exhaustive(D, ids, dist, sel, k):
    oi, od = par_knn(D["Vq"][list(sel)], D["Vs"], k)
    ids_h, dist_h = ids.cpu().numpy(), dist.cpu().numpy()
    for i, q in enumerate(sel):
        np.testing.assert_array_equal(ids_h[q], oi[i], err_msg=f"ids of query {q}")
        np.testing.assert_array_equal(dist_h[q], od[i], err_msg=f"Delta of query {q}")


def test_10m_768_popcount_scan_exhaustive(evp_lib, dev, db_10m_768):
    D = db_10m_768
    st = evp_lib.new_status(dev)
    Tq = evp_lib.encode(D["Q"][:40].contiguous(), D["x"], status=st)
    ids, dist = evp_lib.ternary_knn(Tq, D["Ts"], D["d"], D["x"], 100, status=st,
                                    path=evp_lib.PATH_POPC)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    _check_exhaustive(D, ids, dist, (0, 15, 16, 31, 39), 100)


def test_10m_768_bench_launch_exhaustive(evp_lib, dev, db_10m_768):
    """The benchmark's step: 1,024 float queries through the resident
    database's search (encode -> fp4 tensor-core scan for the shortlist of
    100 -> rerank to 10), plus the plain kNN of the same launch."""
    D = db_10m_768
    n_sl, k = 100, 10
    st = evp_lib.new_status(dev)
    db = evp_lib.Database(D["Ts"], D["U"], D["d"], D["x"])
    Tq = evp_lib.encode(D["Q"], D["x"], status=st)
    sl, sd = db.knn(Tq, n_sl, status=st, path=evp_lib.PATH_MMA)
    sl_a, sd_a = db.knn(Tq, n_sl, status=st)       # the automatic choice (fp4 here)
    rid, rsc = db.search(D["Q"], n_sl, k, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert torch.equal(sl, sl_a) and torch.equal(sd, sd_a)
    # query tiles 0, 1, 3 and 7; lanes of every epilogue warp; both CTAs of a pair
    sel = (0, 1, 127, 128, 129, 383, 511, 640, 1023)
    _check_exhaustive(D, sl, sd, sel, n_sl)
    sl_h, rid_h, rsc_h = sl.cpu().numpy(), rid.cpu().numpy(), rsc.cpu().numpy()
    for q in sel[:4]:
        rows = D["U"][torch.from_numpy(sl_h[q]).to(dev)].cpu().numpy()
        g_local = np.array([[int(np.where(sl_h[q] == j)[0][0]) for j in rid_h[q]]])
        local = np.arange(n_sl, dtype=np.int64)[None, :]
        check_rerank(g_local, rsc_h[q:q + 1], D["Q_h"][q:q + 1], rows, local, k)
    db.close()


@pytest.mark.parametrize("nq", [16, 64])
def test_10m_768_packed_scan_exhaustive(evp_lib, dev, db_10m_768, nq):
    D = db_10m_768
    st = evp_lib.new_status(dev)
    Tq = evp_lib.encode(D["Q"][:nq].contiguous(), D["x"], status=st)
    ids, dist = evp_lib.ternary_knn(Tq, D["Ts"], D["d"], D["x"], 100, status=st,
                                    path=evp_lib.PATH_MMA_PACKED)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    sel = (0, 7, 15) if nq == 16 else (0, 31, 32, 63)
    _check_exhaustive(D, ids, dist, sel, 100)


def test_dense_contraction_10m_1024(evp_lib, dev):
    """10M x 1024, x = 256, 4,096 queries: every code compared with the
    oracle's; the tensor-core scan's shortlist compared with the oracle's
    exhaustive kNN over all 10M rows on queries of several tiles and both
    CTAs of a pair, the popcount scan likewise; the batch also checked
    through the sampled-row properties and its rerank against float64."""
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
    pi, pd = evp_lib.ternary_knn(Tq[:6].contiguous(), Ts, d, x, n_sl, status=st,
                                 path=evp_lib.PATH_POPC)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    # every code, and the exhaustive kNN over all rows
    U_h = U.cpu().numpy()
    Vs = par_encode(U_h, x)
    del U_h
    np.testing.assert_array_equal(_host_codes(Ts), par_pack(Vs))
    Q_h_all = Q.cpu().numpy()
    ex_sel = (0, 127, 128, 129, 2047, 2048, 4095)
    oi, od = par_knn(oracle.encode(Q_h_all[list(ex_sel)], x), Vs, n_sl)
    sl_all, sd_all = sl.cpu().numpy(), sd.cpu().numpy()
    for i, q in enumerate(ex_sel):
        np.testing.assert_array_equal(sl_all[q], oi[i], err_msg=f"ids of query {q}")
        np.testing.assert_array_equal(sd_all[q], od[i], err_msg=f"Delta of query {q}")
    for q in (0, 5):
        np.testing.assert_array_equal(pi.cpu().numpy()[q], sl_all[q])
        np.testing.assert_array_equal(pd.cpu().numpy()[q], sd_all[q])
    del Vs
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
