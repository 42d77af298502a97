"""evp_encode on the GPU against the oracle: packed codes bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00528_gb300 import synth

pytestmark = pytest.mark.gpu


def _gpu_codes(evp, U_np, x, dev):
    st = evp.new_status(dev)
    T = evp.encode(torch.from_numpy(U_np).to(dev), x, status=st)
    torch.cuda.synchronize()
    return T.cpu().numpy().view(np.uint64), int(st.item())


@pytest.mark.parametrize("d", [1, 2, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 384, 500, 768,
                               1000, 1024, 1500, 2048])
def test_encode_matches_oracle_across_d(evp_lib, dev, d):
    U = synth.mixture_numpy(777, d, n_centres=8, anisotropic=d > 8, stream=100 + d)
    xs = sorted({1, max(1, d // 3), oracle.default_x(d), max(1, d - 1), d})
    for x in xs:
        T, st = _gpu_codes(evp_lib, U, x, dev)
        assert st == 0
        np.testing.assert_array_equal(T, oracle.pack(oracle.encode(U, x)), err_msg=f"d={d} x={x}")


def test_encode_ties_zeros_and_signed_zero(evp_lib, dev):
    rng = np.random.default_rng(7)
    d = 384
    # heavily quantised values: many equal magnitudes, both signs, zeros
    U = (rng.integers(-3, 4, size=(500, d)) * 0.125).astype(np.float32)
    U[0] = 0.0
    U[1] = -0.0
    U[2, ::2] = -0.0
    U[3] = 0.5
    U[4, :] = np.where(np.arange(d) % 2 == 0, 0.25, -0.25)
    for x in (1, 37, 128, 256, 383, 384):
        T, st = _gpu_codes(evp_lib, U, x, dev)
        assert st == 0
        np.testing.assert_array_equal(T, oracle.pack(oracle.encode(U, x)), err_msg=f"x={x}")


def test_encode_worked_example(evp_lib, dev):
    from conftest import read_golden
    g = read_golden("table3_worked_example.txt")
    U = np.array([[float(v) for v in g["u1"]], [float(v) for v in g["u2"]]], dtype=np.float32)
    T, st = _gpu_codes(evp_lib, U, 5, dev)
    V, bad = oracle.unpack(T, 10)
    assert bad == 0 and st == 0
    assert V[0].tolist() == [int(v) for v in g["v1_printed"]]
    assert V[1].tolist() == [int(v) for v in g["v2_rule"]]


def test_encode_nonfinite_sets_status(evp_lib, dev):
    U = synth.mixture_numpy(64, 100, stream=5)
    U[17, 3] = np.nan
    _, st = _gpu_codes(evp_lib, U, 67, dev)
    assert st == evp_lib.EVP_ERR_NONFINITE
    U[17, 3] = np.inf
    _, st = _gpu_codes(evp_lib, U, 67, dev)
    assert st == evp_lib.EVP_ERR_NONFINITE
    U[17, 3] = 0.1
    _, st = _gpu_codes(evp_lib, U, 67, dev)
    assert st == 0


def test_encode_empty_and_single_row(evp_lib, dev):
    U = np.zeros((0, 64), dtype=np.float32)
    T = evp_lib.encode(torch.from_numpy(U).to(dev), 3)
    assert T.shape == (0, 2)
    U = synth.mixture_numpy(1, 700, stream=6)
    T, st = _gpu_codes(evp_lib, U, 467, dev)
    np.testing.assert_array_equal(T, oracle.pack(oracle.encode(U, 467)))


def test_encode_argument_errors(evp_lib, dev):
    U = torch.zeros((4, 16), device=dev)
    with pytest.raises(evp_lib.EvpError):
        evp_lib.encode(U, 17)
    with pytest.raises(evp_lib.EvpError):
        evp_lib.encode(torch.zeros((4, 4096), device=dev), 5)
