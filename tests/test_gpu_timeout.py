"""Failure detection on the GPU without a fault: a tensor-core scan whose
copy producer stalls (evp_test_stall_producer) must give up after its
bounded waits, report EVP_ERR_TIMEOUT in the status word, drain what it had
issued, free its tensor memory and leave the device usable -- the next
calls return the oracle's results."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth

pytestmark = pytest.mark.gpu


def _case(evp, dev, ns, nq, d, x, stream):
    U = synth.mixture_numpy(ns, d, n_centres=32, stream=stream)
    Qf = synth.mixture_numpy(nq, d, n_centres=32, stream=stream + 1)
    S = evp.encode(torch.from_numpy(U).to(dev), x)
    Q = evp.encode(torch.from_numpy(Qf).to(dev), x)
    return U, Qf, S, Q


@pytest.mark.parametrize("path,nq,fills", [
    (2, 300, 0),     # fp4 tensor-core scan (CTA pairs): first CTA issues nothing
    (2, 300, 7),     # ... stalls mid-tile, its pair peer has issued more
    (3, 16, 0),      # packed tensor-core scan
    (3, 40, 5),
])
def test_stalled_producer_times_out_and_device_recovers(evp_lib, dev, path, nq, fills):
    d, x, k, ns = 384, 128, 20, 200_000
    U, Qf, S, Q = _case(evp_lib, dev, ns, nq, d, x, 700 + path)
    st = evp_lib.new_status(dev)
    evp_lib.test_stall_producer(path, fills)
    evp_lib.ternary_knn(Q, S, d, x, k, status=st, path=path)
    torch.cuda.synchronize()
    assert int(st.item()) == evp_lib.EVP_ERR_TIMEOUT
    # the stall was one-shot: the same call now completes and is exact
    st2 = evp_lib.new_status(dev)
    ids, dist = evp_lib.ternary_knn(Q, S, d, x, k, status=st2, path=path)
    torch.cuda.synchronize()
    assert int(st2.item()) == 0
    sel = [0, nq // 2, nq - 1]
    Vq = oracle.encode(Qf[sel], x)
    Vs = oracle.encode(U, x)
    oi, od = oracle.knn(Vq, Vs, k)
    np.testing.assert_array_equal(ids.cpu().numpy()[sel], oi)
    np.testing.assert_array_equal(dist.cpu().numpy()[sel], od)


def test_stall_hook_rejects_other_paths(evp_lib):
    with pytest.raises(evp_lib.EvpError) as e:
        evp_lib.test_stall_producer(evp_lib.PATH_POPC, 3)
    assert e.value.code == evp_lib.EVP_ERR_INVALID
