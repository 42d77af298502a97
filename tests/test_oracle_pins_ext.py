"""Pins of the oracle functions for the asymmetric (int8-query) search, the
sparse small-x code and the float32 Euclidean baseline -- each checked
against something other than its own formula: the paper's worked example,
library routines, closed forms, invariants and brute force."""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2506_00528_gb300 import synth


# ---- quantize_i8: symmetric per-query int8 (reading of Sec. 6) ----------

def test_quantize_keeps_integer_vectors_exactly():
    # q = c * n with n integer, max |n| = 127 and c a power of two: the scale
    # 127 / (127 c) = 1 / c is exact, so the integers come back unchanged
    rng = np.random.default_rng(1)
    for c in (1.0, 0.25, 2.0 ** -9, 8.0):
        n = rng.integers(-127, 128, size=(20, 37))
        n[:, 5] = 127
        n[::2, 5] = -127
        q8 = oracle.quantize_i8((n * c).astype(np.float32))
        np.testing.assert_array_equal(q8, n)


def test_quantize_rounds_half_to_even():
    q = np.array([[127.0, 2.5, 3.5, -2.5, -3.5, 0.5, -0.5, 1.5, 126.5]], dtype=np.float32)
    np.testing.assert_array_equal(oracle.quantize_i8(q), [[127, 2, 4, -2, -4, 0, 0, 2, 126]])


def test_quantize_bounds_and_invariants():
    rng = np.random.default_rng(2)
    Q = rng.standard_normal((50, 300)).astype(np.float32)
    q8 = oracle.quantize_i8(Q).astype(np.int64)
    m = np.abs(Q.astype(np.float64)).max(axis=1, keepdims=True)
    exact = Q.astype(np.float64) * 127.0 / m
    assert np.all(np.abs(q8 - exact) <= 0.5 + 1e-4)          # round to nearest
    assert np.all(np.abs(q8).max(axis=1) == 127)             # the largest maps to +-127
    np.testing.assert_array_equal(oracle.quantize_i8(-Q), -q8)   # odd symmetry
    np.testing.assert_array_equal(oracle.quantize_i8(Q * np.float32(4.0)), q8)  # scale
    np.testing.assert_array_equal(oracle.quantize_i8(np.zeros((2, 9), np.float32)),
                                  np.zeros((2, 9), np.int8))


def test_quantize_rejects_nonfinite():
    Q = np.ones((2, 8), dtype=np.float32)
    Q[1, 3] = np.nan
    with pytest.raises(oracle.NonFiniteInput):
        oracle.quantize_i8(Q)
    Q[1, 3] = np.inf
    with pytest.raises(oracle.NonFiniteInput):
        oracle.quantize_i8(Q)


# ---- masked addition and the search by it (Sec. 5.1.2, Sec. 6) ----------

@pytest.mark.parametrize("d,x", [(10, 5), (100, 67), (384, 128), (768, 512)])
def test_masked_sum_is_the_scalar_product(d, x):
    # masked addition computes <q, v> without multiplications (Sec. 5.1.2):
    # compare with numpy's integer dot product
    V = synth.ternary_random(30, d, x, stream=21)
    rng = np.random.default_rng(d)
    Q8 = rng.integers(-127, 128, size=(30, d)).astype(np.int8)
    for i in range(30):
        assert oracle.masked_sum(Q8[i], V[i]) == int(np.dot(Q8[i].astype(np.int64),
                                                            V[i].astype(np.int64)))


def test_masked_sum_of_a_ternary_query_is_b2sp():
    # a query that is itself a ternary code: masked addition = b2sp, the
    # paper's four-term bitplane count (Sec. 5.1.2)
    d, x = 100, 40
    V = synth.ternary_random(20, d, x, stream=22)
    T = oracle.pack(V)
    W = oracle.words(d)

    def bsp(a, b):
        return sum(bin(int(a[i]) & int(b[i])).count("1") for i in range(W))

    for i in range(0, 20, 2):
        t1, t2 = T[i], T[i + 1]
        b2sp = bsp(t1[:W], t2[:W]) + bsp(t1[W:], t2[W:]) - bsp(t1[:W], t2[W:]) - bsp(t1[W:], t2[:W])
        assert oracle.masked_sum(V[i], V[i + 1]) == b2sp


def test_knn_i8q_bruteforce_with_planted_ties():
    d, x, ns = 24, 9, 60
    V = synth.ternary_random(ns, d, x, stream=23)
    V[10] = V[3]           # exact duplicates tie on every query
    V[41] = V[3]
    V[55] = V[20]
    rng = np.random.default_rng(3)
    Q8 = rng.integers(-127, 128, size=(7, d)).astype(np.int8)
    for k in (1, 5, 17, ns):
        ids, sc = oracle.knn_i8q(Q8, V, k)
        for q in range(7):
            scores = [sum(int(Q8[q, j]) * int(V[s, j]) for j in range(d)) for s in range(ns)]
            order = sorted(range(ns), key=lambda s: (-scores[s], s))[:k]
            assert ids[q].tolist() == order
            assert sc[q].tolist() == [scores[s] for s in order]


def test_knn_i8q_of_ternary_queries_orders_as_delta():
    # for a ternary query with x non-zeros, Delta = 2x - 2 <q, s>: the search
    # by masked addition returns the Delta search's list
    d, x, ns, k = 64, 30, 500, 25
    V = synth.ternary_random(ns, d, x, stream=24)
    Vq = synth.ternary_random(6, d, x, stream=25)
    i1, s1 = oracle.knn_i8q(Vq, V, k)
    i2, d2 = oracle.knn(Vq, V, k)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_array_equal(2 * x - 2 * s1.astype(np.int64), d2)


# ---- sparse index-list code (Sec. 6, different EVPs) ----------------------

def _entries(tokens):
    out = []
    for t in tokens:
        out.append(0x8000 | int(t[1:]) if t.startswith("-") else int(t))
    return np.array(out, dtype=np.uint16)


def test_sparse_code_of_the_worked_example():
    g = read_golden("table3_worked_example.txt")
    s = read_golden("table3_sparse_codes.txt")
    x, d = int(g["x"][0]), int(g["d"][0])
    v1 = np.array([[int(t) for t in g["v1_printed"]]], dtype=np.int8)
    v2 = np.array([[int(t) for t in g["v2_rule"]]], dtype=np.int8)
    np.testing.assert_array_equal(oracle.sparse_pack(v1, x)[0], _entries(s["v1_sparse"]))
    np.testing.assert_array_equal(oracle.sparse_pack(v2, x)[0], _entries(s["v2_rule_sparse"]))
    # and the encoder's own output, from the printed floats
    u1 = np.array([[float(t) for t in g["u1"]]], dtype=np.float32)
    np.testing.assert_array_equal(oracle.sparse_pack(oracle.encode(u1, x), x)[0],
                                  _entries(s["v1_sparse"]))
    V, bad = oracle.sparse_unpack(_entries(s["v2_rule_sparse"])[None], d)
    assert bad == 0
    np.testing.assert_array_equal(V, v2)


@pytest.mark.parametrize("d,x", [(10, 5), (768, 64), (1024, 32), (300, 300)])
def test_sparse_round_trip_and_order(d, x):
    V = synth.ternary_random(50, d, x, stream=26)
    E = oracle.sparse_pack(V, x)
    dims = (E & 0x7FFF).astype(np.int64)
    assert np.all(np.diff(dims, axis=1) > 0)                   # strictly ascending
    neg = (E & 0x8000) != 0
    rows = np.arange(50)[:, None]
    assert np.all(V[rows, dims] == np.where(neg, -1, 1))        # sign bit = -1
    V2, bad = oracle.sparse_unpack(E, d)
    assert bad == 0
    np.testing.assert_array_equal(V2, V)


def test_sparse_rejects_malformed():
    V = synth.ternary_random(3, 20, 4, stream=27)
    with pytest.raises(ValueError):
        oracle.sparse_pack(V, 5)                                # wrong count
    E = oracle.sparse_pack(V, 4)
    E[1, 2] = E[1, 1]                                           # repeated dimension
    E[2, 3] = 25                                                # dimension >= d
    _, bad = oracle.sparse_unpack(E, 20)
    assert bad == 2


# ---- float32 Euclidean brute force (the paper's float baseline) ----------

def test_l2_knn_matches_float64_within_rounding():
    rng = np.random.default_rng(4)
    d, ns, nq, k = 96, 3000, 6, 20
    S = rng.standard_normal((ns, d)).astype(np.float32)
    Q = rng.standard_normal((nq, d)).astype(np.float32)
    S[100] = S[7]                                              # exact tie: lower index first
    ids, dist = oracle.l2_knn(Q, S, k)
    D64 = ((Q.astype(np.float64)[:, None, :] - S.astype(np.float64)[None]) ** 2).sum(-1)
    for q in range(nq):
        exact = D64[q, ids[q]]
        # float32 sum of d non-negative terms: relative error <= d * 2^-24 (with margin)
        assert np.all(np.abs(dist[q] - exact) <= 2 * d * 2.0 ** -24 * exact + 1e-30)
        ref = np.argsort(D64[q], kind="stable")[:k]
        kth = D64[q, ref[-1]]
        gap = 4 * d * 2.0 ** -24 * kth
        clear = [i for i in ref if D64[q, i] < kth - gap]
        assert set(clear) <= set(ids[q].tolist())
    _, d7 = oracle.l2_knn(S[7:8], S, 3)
    i7, _ = oracle.l2_knn(S[7:8], S, 2)
    assert i7[0].tolist() == [7, 100] and d7[0, 0] == 0.0 and d7[0, 1] == 0.0
