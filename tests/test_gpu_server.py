"""Continuous-batching server: every request's result is bit-identical to
the same request run alone through evp_db_search_host, and agrees with the
oracle (exhaustive shortlist by Delta, float64 rerank); admission by memory;
a stalled worker (paused on the host) makes waits time out."""
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth
from test_gpu_rerank import check_rerank

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served_db(dev, evp_lib):
    d, x = 384, 128
    U = synth.mixture_numpy(20_000, d, n_centres=64, stream=synth.STREAM_DB)
    Ud = torch.from_numpy(U).to(dev)
    T = evp_lib.encode(Ud, x)
    db = evp_lib.Database(T, Ud, d, x)
    db.U_host, db.V_oracle = U, oracle.encode(U, x)
    yield db
    db.close()


def _alone(evp_lib, db, Q, k, factor):
    n_sl = min(factor * k, 1024)
    ids = torch.empty((Q.shape[0], k), dtype=torch.int64).pin_memory()
    sc = torch.empty((Q.shape[0], k), dtype=torch.float32).pin_memory()
    st = evp_lib.new_status("cuda")
    db.search_host(torch.from_numpy(Q).pin_memory(), n_sl, k, ids, sc, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return ids.clone(), sc.clone()


def test_mixed_requests_match_alone(evp_lib, served_db):
    rng = np.random.default_rng(3)
    Qall = synth.mixture_numpy(3000, 384, n_centres=64, stream=synth.STREAM_QUERIES)
    reqs = []
    off = 0
    for i in range(60):
        nq = int(rng.integers(1, 80))
        k = int(rng.choice([5, 20]))
        reqs.append((Qall[off:off + nq].copy(), k))
        off += nq
    srv = evp_lib.Server(served_db, max_batch_queries=256, max_k=20, shortlist_factor=10,
                         max_slots=3, mem_budget_bytes=8 << 30)
    assert srv.slots == 3
    rids = [None] * len(reqs)

    def producer(lo, hi):
        for i in range(lo, hi):
            rids[i] = srv.submit(reqs[i][0], reqs[i][1])

    th = [threading.Thread(target=producer, args=(j * 15, (j + 1) * 15)) for j in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    out = [srv.wait(r, timeout_s=60) for r in rids]
    stats = srv.stats()
    srv.close()
    assert stats["requests"] == len(reqs) and stats["p99_us"] >= stats["p50_us"] > 0
    assert stats["batches"] < len(reqs)            # requests were coalesced
    for i, ((Q, k), (ids, sc, status, lat)) in enumerate(zip(reqs, out)):
        assert status == 0 and lat > 0
        ai, asc = _alone(evp_lib, served_db, Q, k, 10)
        assert torch.equal(ids, ai)
        assert torch.equal(sc, asc)
        if i % 4 == 0:
            # the oracle: exhaustive shortlist of 10 k by Delta, float64 rerank to k
            sl, _ = oracle.knn(oracle.encode(Q, served_db.x), served_db.V_oracle, 10 * k)
            check_rerank(ids.numpy(), sc.numpy(), Q, served_db.U_host, sl, k)


def test_admission_by_memory(evp_lib, served_db):
    # a budget below one slot's workspace admits nothing
    with pytest.raises(evp_lib.EvpError) as e:
        evp_lib.Server(served_db, max_batch_queries=1024, max_k=20, mem_budget_bytes=1024)
    assert e.value.code == evp_lib.EVP_ERR_NO_MEMORY
    # the slot count follows the budget: a budget for about two slots gives two
    probe = evp_lib.Server(served_db, max_batch_queries=128, max_k=20, max_slots=1,
                           mem_budget_bytes=8 << 30)
    probe.close()
    per_slot = max(int(evp_lib.load().evp_db_search_host_workspace(
        served_db.handle, 128, min(10 * k, 1024), k)) for k in range(1, 21))
    srv = evp_lib.Server(served_db, max_batch_queries=128, max_k=20, max_slots=8,
                         mem_budget_bytes=int(2.5 * (per_slot + 256)))
    assert srv.slots == 2
    # a request larger than a slot is refused at submission
    with pytest.raises(evp_lib.EvpError) as e:
        srv.submit(synth.mixture_numpy(200, 384, stream=31), 5)
    assert e.value.code == evp_lib.EVP_ERR_NO_MEMORY
    srv.close()


def test_stalled_worker_times_out_then_recovers(evp_lib, served_db):
    srv = evp_lib.Server(served_db, max_batch_queries=64, max_k=20, max_slots=2,
                         mem_budget_bytes=8 << 30)
    srv.pause(True)
    Q = synth.mixture_numpy(8, 384, stream=32)
    rid = srv.submit(Q, 5)
    with pytest.raises(evp_lib.EvpError) as e:
        srv.wait(rid, timeout_s=0.2)
    assert e.value.code == evp_lib.EVP_ERR_TIMEOUT
    srv.pause(False)
    ids, sc, status, _ = srv.wait(rid, timeout_s=30)
    assert status == 0
    ai, asc = _alone(evp_lib, served_db, Q, 5, 10)
    assert torch.equal(ids, ai) and torch.equal(sc, asc)
    srv.close()
