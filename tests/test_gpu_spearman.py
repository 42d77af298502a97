"""Table 1's 'Uniform' rows through the library (the correlation study of
Sec. 5.2): the proxy distances the GPU scan returns for all query x
database pairs equal the oracle's Delta, and their Spearman correlation with
the true Euclidean distance orders EVP > b1.58 > 1-bit, with EVP close to
the printed 0.80 (d = 100) and 0.79 (d = 1000)."""
import os
import sys

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,rho_paper", [(100, 0.80), (1000, 0.79)])
def test_spearman_through_the_library(evp_lib, dev, d, rho_paper):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2506_00528_gb300 import synth
    r = bench.spearman_study(evp_lib, synth, dev, d)
    nq = r["D_evp"].shape[0]
    U = synth.uniform_sphere(nq + r["D_evp"].shape[1], d, stream=30 + d)
    V = oracle.encode(U, r["x"]).astype(np.int64)
    ref = ((V[:nq, None, :] - V[None, nq:, :]) ** 2).sum(-1)
    np.testing.assert_array_equal(r["D_evp"], ref)
    assert r["rho_evp"] > r["rho_b158"] > r["rho_1bit"]
    assert abs(r["rho_evp"] - rho_paper) < 0.05, r["rho_evp"]
