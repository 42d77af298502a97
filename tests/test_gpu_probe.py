"""The tensor-core rate probe (measurement support): it runs on every SM,
reports plausible rates, e4m3 instructions (K = 32) deliver about twice the
flops of bf16 ones (K = 16) at the same shape, and block-scaled fp4
instructions (kind::mxf4, K = 64) about twice those of e4m3."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_rates(evp_lib, dev):
    f8, c8, ms8 = evp_lib.probe_tensor_rate(kind=0, cta_pair=False, n=256, iters=1 << 14)
    f8p, c8p, _ = evp_lib.probe_tensor_rate(kind=0, cta_pair=True, n=256, iters=1 << 14)
    bf, cb, _ = evp_lib.probe_tensor_rate(kind=1, cta_pair=False, n=256, iters=1 << 14)
    f4, c4, _ = evp_lib.probe_tensor_rate(kind=2, cta_pair=False, n=256, iters=1 << 14)
    f4p, c4p, _ = evp_lib.probe_tensor_rate(kind=2, cta_pair=True, n=256, iters=1 << 14)
    for v in (f8, f8p, bf, f4, f4p):
        assert 100.0 < v < 40000.0
    for c in (c8, c8p, cb, c4, c4p):
        assert 32.0 < c < 4096.0
    assert f8 > 1.5 * bf
    assert f4 > 1.5 * f8 and f4p > 1.5 * f8p
    _, c16, _ = evp_lib.probe_tensor_rate(kind=0, cta_pair=False, n=16, iters=1 << 14)
    assert c16 <= c8


def test_probe_argument_checks(evp_lib, dev):
    for kw in ({"kind": 3}, {"kind": 2 | 0x400}, {"kind": 2 | 0x100}, {"kind": 1 | 0x1000},
               {"n": 8}, {"n": 264}, {"n": 24}, {"iters": 0}):
        args = {"kind": 0, "cta_pair": False, "n": 256, "iters": 16}
        args.update(kw)
        with pytest.raises(evp_lib.EvpError) as e:
            evp_lib.probe_tensor_rate(**args)
        assert e.value.code == evp_lib.EVP_ERR_INVALID
