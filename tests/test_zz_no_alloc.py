"""ternary_knn_static -- the entry point that allocates nothing -- against
the workspace-taking ternary_knn (popcount path), on two calls in a row.

It is for callers that cannot allocate device memory (serving threads that
must stay out of the device allocator, plugins and plain C callers handed
raw pointers); its scratch is a fixed array inside the library.  The file is
named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2506_00528_gb300 import synth

pytestmark = pytest.mark.gpu


def _codes(evp, n, d, x, stream, dev):
    U = torch.from_numpy(synth.mixture_numpy(n, d, n_centres=32, stream=stream)).to(dev)
    return evp.encode(U, x)


def test_static_scratch_matches_ternary_knn_twice(evp_lib, dev):
    d, x, k = 384, 128, 50
    S = _codes(evp_lib, 30_000, d, x, 900, dev)
    for call, (nq, qstream) in enumerate([(37, 901), (16, 902)]):
        Q = _codes(evp_lib, nq, d, x, qstream, dev)
        st = evp_lib.new_status(dev)
        ref_ids, ref_dist = evp_lib.ternary_knn(Q, S, d, x, k, status=st, path=evp_lib.PATH_POPC)
        ids = torch.full((nq, k), -7, dtype=torch.int64, device=dev)
        dist = torch.full((nq, k), -7, dtype=torch.int32, device=dev)
        evp_lib.ternary_knn_static(Q, S, d, x, k, ids, dist, status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0, call
        assert torch.equal(ids, ref_ids), call
        assert torch.equal(dist, ref_dist), call


def test_static_scratch_rejects_oversized_requests(evp_lib, dev):
    d, x = 64, 40
    S = _codes(evp_lib, 200_000, d, x, 903, dev)
    Q = _codes(evp_lib, 4, d, x, 904, dev)
    k = 1024   # popcount-path workspace above the 16 MiB scratch
    need = evp_lib.knn_workspace_bytes(4, 200_000, d, k, evp_lib.PATH_POPC)
    assert need > (16 << 20)
    ids = torch.empty((4, k), dtype=torch.int64, device=dev)
    dist = torch.empty((4, k), dtype=torch.int32, device=dev)
    with pytest.raises(evp_lib.EvpError) as e:
        evp_lib.ternary_knn_static(Q, S, d, x, k, ids, dist)
    assert e.value.code == evp_lib.EVP_ERR_NO_MEMORY


def test_static_binding_rejects_wrong_outputs(evp_lib, dev):
    """The outputs are the caller's: a wrong shape, dtype or device is
    refused on the host before anything is launched."""
    d, x, k = 128, 40, 10
    S = _codes(evp_lib, 2_000, d, x, 905, dev)
    Q = _codes(evp_lib, 5, d, x, 906, dev)
    ok_i = torch.empty((5, k), dtype=torch.int64, device=dev)
    ok_d = torch.empty((5, k), dtype=torch.int32, device=dev)
    bad = [
        (torch.empty((5, k - 1), dtype=torch.int64, device=dev), ok_d),   # too small
        (torch.empty((4, k), dtype=torch.int64, device=dev), ok_d),
        (torch.empty((5, k), dtype=torch.int32, device=dev), ok_d),       # wrong dtype
        (ok_i, torch.empty((5, k), dtype=torch.int64, device=dev)),
        (torch.empty((5, k), dtype=torch.int64), ok_d),                   # host tensor
    ]
    for ids, dist in bad:
        with pytest.raises(ValueError):
            evp_lib.ternary_knn_static(Q, S, d, x, k, ids, dist)
    evp_lib.ternary_knn_static(Q, S, d, x, k, ok_i, ok_d)
    torch.cuda.synchronize()
