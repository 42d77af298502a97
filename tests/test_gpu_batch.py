"""Batched form: uneven batches against three resident databases, planned
once (autotuned paths), run eagerly and as a captured CUDA graph; every
batch equals its own evp_db_search / evp_db_knn call, the fused multi-batch
tensor-core scan equals the batches run separately, and every batch agrees
with the oracle (exhaustive kNN by Delta; float64 rerank of the shortlist)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth
from test_gpu_rerank import check_rerank

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbs(dev, evp_lib):
    out = []
    for i, (n, d, x) in enumerate([(20_000, 384, 128), (30_000, 768, 256), (15_000, 1024, 384)]):
        U = torch.from_numpy(synth.mixture_numpy(n, d, n_centres=32, anisotropic=True,
                                                 stream=1000 + i)).to(dev)
        T = evp_lib.encode(U, x)
        out.append((evp_lib.Database(T, U, d, x), U, d, x))
    yield out
    for db, *_ in out:
        db.close()


def _batches(evp_lib, dbs, dev):
    sizes = [1, 5, 17, 200, 3, 64, 129, 1, 31, 400, 16, 2]
    spec = []
    for i, nq in enumerate(sizes):
        db, U, d, x = dbs[i % 3]
        Q = torch.from_numpy(synth.mixture_numpy(nq, d, n_centres=32, anisotropic=True,
                                                 stream=2000 + i)).to(dev)
        if i % 4 == 3:    # plain kNN on packed codes
            spec.append({"db": db, "Qc": evp_lib.encode(Q, x), "k": 100 if i % 8 == 3 else 10})
        else:             # whole path: shortlist 10k, rerank to k
            k = 10 if i % 2 else 5
            spec.append({"db": db, "Q": Q, "n_shortlist": 10 * k, "k": k})
    return spec


def _alone(evp_lib, b):
    if "Q" in b:
        return b["db"].search(b["Q"], b["n_shortlist"], b["k"])
    return b["db"].knn(b["Qc"], b["k"])


@pytest.mark.parametrize("graph,tune", [(True, True), (False, False)])
def test_batch_plan_matches_per_batch_calls(evp_lib, dev, dbs, graph, tune):
    spec = _batches(evp_lib, dbs, dev)
    stream = torch.cuda.Stream()
    plan = evp_lib.BatchPlan(spec, graph=graph, tune=tune, stream=stream)
    for i in range(len(spec)):
        assert plan.path(i) in ((1, 2, 3) if tune else (0,))
    st = evp_lib.new_status(dev)
    with torch.cuda.stream(stream):
        plan.run(status=st, stream=stream)     # capture (graph) or eager
    stream.synchronize()
    first = [tuple(t.clone() for t in plan.outputs(i)) for i in range(len(spec))]
    for o in plan.outputs(0):
        o.fill_(-9)
    with torch.cuda.stream(stream):
        plan.run(status=st, stream=stream)     # replay
    stream.synchronize()
    assert int(st.item()) == 0
    for i, b in enumerate(spec):
        ref = _alone(evp_lib, b)
        torch.cuda.synchronize()
        got = plan.outputs(i)
        for r, g, f in zip(ref, got, first[i]):
            assert torch.equal(r, g), i
            assert torch.equal(r, f), i
    plan.close()


def test_autotune_caches_and_reports(evp_lib, dbs):
    db = dbs[1][0]
    evp_lib.load().evp_autotune_clear()
    path, pm, mm = evp_lib.autotune(db, 256, 10, measure=True)
    assert path in (1, 2, 3) and pm > 0 and mm > 0
    assert (path == 1) == (pm <= mm)
    assert evp_lib.autotune(db, 200, 10)[0] == path     # same bucket -> cached
    path_big_k, pm2, mm2 = evp_lib.autotune(db, 40, 500, measure=True)
    assert (path_big_k == 1) == (pm2 <= mm2)


def _oracle_check(spec, dbs, outs):
    hosts = {id(db): (U.cpu().numpy(), x) for db, U, d, x in dbs}
    for b, (ids, second) in zip(spec, outs):
        U, x = hosts[id(b["db"])]
        V = oracle.encode(U, x)
        if "Q" in b:
            Q = b["Q"].cpu().numpy()
            sl, _ = oracle.knn(oracle.encode(Q, x), V, b["n_shortlist"])
            check_rerank(ids.cpu().numpy(), second.cpu().numpy(), Q, U, sl, b["k"])
        else:
            d = U.shape[1]
            Vq, bad = oracle.unpack(b["Qc"].cpu().numpy().view(np.uint64), d)
            assert bad == 0
            oi, od = oracle.knn(Vq, V, b["k"])
            np.testing.assert_array_equal(ids.cpu().numpy(), oi)
            np.testing.assert_array_equal(second.cpu().numpy(), od)


@pytest.mark.parametrize("graph,tune", [(True, False), (False, False), (True, True)])
def test_fused_plan_matches_separate_and_oracle(evp_lib, dev, dbs, graph, tune):
    spec = _batches(evp_lib, dbs, dev)
    stream = torch.cuda.Stream()
    fused = evp_lib.BatchPlan(spec, graph=graph, tune=tune, fused=True, stream=stream)
    sep = evp_lib.BatchPlan(spec, graph=False, tune=tune, fused=False, stream=stream)
    assert sep.fused == 0
    if not tune:
        assert fused.fused == 6          # the batches the automatic rule gives the fp4 scan
    st = evp_lib.new_status(dev)
    with torch.cuda.stream(stream):
        fused.run(status=st, stream=stream)
        sep.run(status=st, stream=stream)
    stream.synchronize()
    for o in fused.outputs(0):
        o.fill_(-9)
    with torch.cuda.stream(stream):
        fused.run(status=st, stream=stream)   # replay (graph) or second eager run
    stream.synchronize()
    assert int(st.item()) == 0
    outs = []
    for i in range(len(spec)):
        a, b = fused.outputs(i), sep.outputs(i)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), i
        assert (fused.tile(i) > 0) == (i in [j for j in range(len(spec)) if fused.tile(j) > 0])
        outs.append(a)
    _oracle_check(spec, dbs, outs)
    fused.close()
    sep.close()


def test_autotune_table_save_and_load(evp_lib, dbs, tmp_path):
    db = dbs[0][0]
    evp_lib.load().evp_autotune_clear()
    path, _, _ = evp_lib.autotune(db, 100, 10, measure=True)
    f = str(tmp_path / "tune.txt")
    evp_lib.autotune_save(f)
    lines = [l for l in open(f) if not l.startswith("#")]
    assert any("|path|384|128|128|10|" in l for l in lines), lines
    evp_lib.load().evp_autotune_clear()
    evp_lib.autotune_load(f)
    assert evp_lib.autotune(db, 100, 10)[0] == path
    with open(f, "a") as fh:
        fh.write("not a line\n")
    with pytest.raises(evp_lib.EvpError):
        evp_lib.autotune_load(f)
