"""ternary_knn on the GPU against the oracle: ids and Delta bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth

pytestmark = pytest.mark.gpu


PATHS = [1, 2, 3]   # EVP_PATH_POPC, EVP_PATH_MMA, EVP_PATH_MMA_PACKED


def packed_supported(d, k):
    """Shapes the packed tensor-core path takes: d <= 768 with an even number
    of 64-bit words per bitplane, k <= 256."""
    W = (d + 63) // 64
    return W % 2 == 0 and W <= 12 and k <= 256


def _run(evp, Tq, Ts, d, x, k, dev, path=0):
    if path in (2, 3) and k > 1024:
        pytest.skip("tensor-core paths take k <= 1024")
    Qd = torch.from_numpy(Tq.view(np.int64)).to(dev)
    Sd = torch.from_numpy(Ts.view(np.int64)).to(dev)
    if path == 3 and not packed_supported(d, k):
        with pytest.raises(evp.EvpError) as e:
            evp.ternary_knn(Qd, Sd, d, x, k, path=path)
        assert e.value.code == evp.EVP_ERR_UNSUPPORTED
        pytest.skip("outside the packed path's shapes (refused as checked)")
    st = evp.new_status(dev)
    ids, dist = evp.ternary_knn(Qd, Sd, d, x, k, status=st, path=path)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return ids.cpu().numpy(), dist.cpu().numpy()


@pytest.mark.parametrize("path", PATHS)
def test_tiny_config_bit_exact(evp_lib, dev, path):
    """The small workload: 10,000 x 384 database, 100 queries, 64-centre
    mixture (sigma 0.5), x = 128, k = 10."""
    d, x, k = 384, 128, 10
    U = synth.mixture_numpy(10_000, d, n_centres=64, stream=synth.STREAM_DB)
    Qf = synth.mixture_numpy(100, d, n_centres=64, stream=synth.STREAM_QUERIES)
    Vs, Vq = oracle.encode(U, x), oracle.encode(Qf, x)
    # codes from the GPU encoder (themselves checked against the oracle)
    st = evp_lib.new_status(dev)
    Ts = evp_lib.encode(torch.from_numpy(U).to(dev), x, status=st)
    Tq = evp_lib.encode(torch.from_numpy(Qf).to(dev), x, status=st)
    ids, dist = evp_lib.ternary_knn(Tq, Ts, d, x, k, status=st, path=path)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    np.testing.assert_array_equal(Ts.cpu().numpy().view(np.uint64), oracle.pack(Vs))
    oi, od = oracle.knn(Vq, Vs, k)
    np.testing.assert_array_equal(ids.cpu().numpy(), oi)
    np.testing.assert_array_equal(dist.cpu().numpy(), od)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("d", [1, 2, 63, 64, 65, 100, 127, 129, 384, 1000, 1024])
def test_shapes_across_d(evp_lib, dev, d, path):
    x = oracle.default_x(d)
    ns = 3001
    Vs = synth.ternary_random(ns, d, x, stream=200 + d)
    Vq = synth.ternary_random(5, d, x, stream=300 + d)
    k = min(50, ns)
    ids, dist = _run(evp_lib, oracle.pack(Vq), oracle.pack(Vs), d, x, k, dev, path)
    oi, od = oracle.knn(Vq, Vs, k)
    np.testing.assert_array_equal(dist, od)
    np.testing.assert_array_equal(ids, oi)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("ns,k", [(1, 1), (255, 255), (256, 17), (257, 257), (1000, 1000),
                                  (5000, 1), (5000, 1024), (70_001, 100),
                                  (70_001, 1024)])
def test_sizes_and_k(evp_lib, dev, ns, k, path):
    d, x = 96, 64
    U = synth.mixture_numpy(ns, d, n_centres=16, stream=400)
    Qf = synth.mixture_numpy(7, d, n_centres=16, stream=401)
    Vs, Vq = oracle.encode(U, x), oracle.encode(Qf, x)
    ids, dist = _run(evp_lib, oracle.pack(Vq), oracle.pack(Vs), d, x, k, dev, path)
    oi, od = oracle.knn(Vq, Vs, k)
    np.testing.assert_array_equal(dist, od)
    np.testing.assert_array_equal(ids, oi)


@pytest.mark.parametrize("path", [0] + PATHS)
@pytest.mark.parametrize("nq", [1, 2, 3, 15, 16, 17, 33, 50, 127, 128, 129, 300])
def test_query_counts_span_passes(evp_lib, dev, nq, path):
    d, x, k = 256, 171, 20
    U = synth.mixture_numpy(20_000, d, n_centres=32, stream=500)
    Qf = synth.mixture_numpy(nq, d, n_centres=32, stream=501)
    Vs, Vq = oracle.encode(U, x), oracle.encode(Qf, x)
    ids, dist = _run(evp_lib, oracle.pack(Vq), oracle.pack(Vs), d, x, k, dev, path)
    oi, od = oracle.knn(Vq, Vs, k)
    np.testing.assert_array_equal(dist, od)
    np.testing.assert_array_equal(ids, oi)


@pytest.mark.parametrize("path,k", [(1, 300), (2, 128), (1, 1024), (2, 300), (2, 1024),
                                    (3, 128), (3, 256), (3, 1024)])
def test_massive_ties(evp_lib, dev, path, k):
    """Only six distinct codes in the database: almost every Delta ties, so
    the (Delta, index) order decides everything, across slices and merges."""
    d, x = 128, 40
    base = synth.ternary_random(6, d, x, stream=600)
    rng = np.random.default_rng(11)
    Vs = base[rng.integers(0, 6, size=60_000)]
    Vq = np.concatenate([base[:3], synth.ternary_random(4, d, x, stream=601)])
    ids, dist = _run(evp_lib, oracle.pack(Vq), oracle.pack(Vs), d, x, k, dev, path)
    oi, od = oracle.knn(Vq, Vs, k)
    np.testing.assert_array_equal(dist, od)
    np.testing.assert_array_equal(ids, oi)


@pytest.mark.parametrize("path,d", [(1, 64), (2, 64), (3, 128)])
def test_identical_database(evp_lib, dev, path, d):
    x = 10
    Vs = np.repeat(synth.ternary_random(1, d, x, stream=602), 9000, axis=0)
    Vq = synth.ternary_random(3, d, x, stream=603)
    ids, dist = _run(evp_lib, oracle.pack(Vq), oracle.pack(Vs), d, x, 64, dev, path)
    assert np.all(ids == np.arange(64)[None, :])
    oi, od = oracle.knn(Vq, Vs[:100], 64)
    np.testing.assert_array_equal(dist, od)


@pytest.mark.parametrize("path,d", [(1, 64), (2, 64), (3, 128)])
def test_descending_stream_worst_case(evp_lib, dev, path, d):
    """Rows ordered so that each is nearer than all earlier ones: every row
    enters the candidate buffers (the merge path under maximum pressure)."""
    x, k = 32, 100
    q = np.zeros((1, d), dtype=np.int8)
    q[0, :32] = 1
    rows = []
    for m in range(33):   # m matching +1 positions, the rest moved out of the query's support
        v = np.zeros(d, dtype=np.int8)
        v[:m] = 1
        v[32:32 + (32 - m)] = 1
        rows.append(v)
    Vs = np.repeat(np.array(rows[::1]), 400, axis=0)      # Delta falls as the index grows
    ids, dist = _run(evp_lib, oracle.pack(q), oracle.pack(Vs), d, x, k, dev, path)
    oi, od = oracle.knn(q, Vs, k)
    np.testing.assert_array_equal(dist, od)
    np.testing.assert_array_equal(ids, oi)


def test_argument_errors(evp_lib, dev):
    Vs = torch.zeros((10, 2), dtype=torch.int64, device=dev)
    with pytest.raises(evp_lib.EvpError):
        evp_lib.ternary_knn(Vs[:1], Vs, 64, 10, 11)            # k > ns
    with pytest.raises(evp_lib.EvpError):
        evp_lib.ternary_knn(Vs[:1], Vs, 64, 65, 3)             # x > d
    big = torch.zeros((10, 34), dtype=torch.int64, device=dev)
    with pytest.raises(evp_lib.EvpError):
        evp_lib.ternary_knn(big[:1], big, 2048, 10, 3)         # d above the scan limit
    with pytest.raises(evp_lib.EvpError):
        evp_lib.ternary_knn(Vs[:1], Vs, 64, 10, 9, path=4)     # unknown path
    with pytest.raises(evp_lib.EvpError):
        evp_lib.ternary_knn(Vs[:1], Vs, 64, 10, 9, path=3)     # packed path: odd word count
    many = torch.zeros((2000, 2), dtype=torch.int64, device=dev)
    with pytest.raises(evp_lib.EvpError):
        evp_lib.ternary_knn(many[:20], many, 64, 10, 1025, path=2)  # k above the limit
    ws = torch.empty(256, dtype=torch.uint8, device=dev)
    out = torch.empty(16, dtype=torch.int64, device=dev)
    rc = evp_lib.load().ternary_knn(Vs.data_ptr(), 1, Vs.data_ptr(), 10, 64, 10, 3,
                                    out.data_ptr(), out.data_ptr(), ws.data_ptr(), 256, None,
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == evp_lib.EVP_ERR_NO_MEMORY


@pytest.mark.parametrize("pair", ["0", "1"])
@pytest.mark.parametrize("nq,ns,d,k", [(1, 3001, 384, 10),      # one tile, the pair's second CTA idle
                                       (129, 70_001, 256, 20),  # two tiles: one pair
                                       (300, 12_000, 768, 10),  # three tiles: odd count
                                       (513, 4_001, 1024, 100),
                                       (100, 40_000, 128, 600),  # qa = 16 queries per tile
                                       (40, 5_000, 64, 1024)])
def test_tensor_path_cta_pair_and_single(evp_lib, dev, monkeypatch, pair, nq, ns, d, k):
    """The tensor-core scan with CTA pairs (M = 256 per instruction, each CTA
    staging half of the database tile) and with single CTAs gives the oracle's
    ids and Delta bit for bit."""
    monkeypatch.setenv("EVP_MMA_CTA_PAIR", pair)
    x = oracle.default_x(d)
    Vs = synth.ternary_random(ns, d, x, stream=900 + d)
    Vq = synth.ternary_random(nq, d, x, stream=950 + d)
    ids, dist = _run(evp_lib, oracle.pack(Vq), oracle.pack(Vs), d, x, k, dev, path=2)
    oi, od = oracle.knn(Vq, Vs, k)
    np.testing.assert_array_equal(dist, od)
    np.testing.assert_array_equal(ids, oi)


@pytest.mark.parametrize("nq,ns,d,k", [(1, 3_001, 768, 10),     # one query: a 16-query pass
                                       (16, 20_000, 768, 100),
                                       (17, 20_000, 768, 100),  # 32-query pass
                                       (64, 50_000, 768, 10),   # one full 64-query pass
                                       (65, 50_000, 768, 10),   # a second pass of one query
                                       (200, 9_000, 384, 50),   # four passes, d = 384
                                       (5, 130_000, 128, 256),
                                       (33, 1_000, 256, 200),
                                       (40, 129, 640, 100)])    # one tile and a ragged row
def test_packed_tensor_path(evp_lib, dev, nq, ns, d, k):
    """The packed tensor-core scan (tiles unpacked on chip, database rows as
    the MMA's M side) gives the oracle's ids and Delta bit for bit, across
    pass sizes, K depths and ragged tiles."""
    x = oracle.default_x(d)
    Vs = synth.ternary_random(ns, d, x, stream=1100 + d)
    Vq = synth.ternary_random(nq, d, x, stream=1150 + d)
    ids, dist = _run(evp_lib, oracle.pack(Vq), oracle.pack(Vs), d, x, k, dev, path=3)
    oi, od = oracle.knn(Vq, Vs, k)
    np.testing.assert_array_equal(dist, od)
    np.testing.assert_array_equal(ids, oi)
