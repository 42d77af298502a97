"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check uses a value printed
in the paper (golden fixtures under tests/golden/, each with its citation), a
closed form, a brute-force enumeration on tiny inputs, an invariant, or an
independent formula (the paper's four-term bitplane definition of b2sp).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2506_00528_gb300 import synth
from conftest import read_golden, read_golden_rows


def _floats(vals):
    return np.array([float(v) for v in vals], dtype=np.float32)


def _ints(vals):
    return np.array([int(v) for v in vals], dtype=np.int8)


# ---------------------------------------------------------------- choice of x


def test_default_x_matches_printed_evps():
    """Table 2 and Table 5 list the EVPs used: {67,100}, {667,1000}, {256,384},
    {333,500}, {512,768} -- each the maximiser of C(d,x)*2^x (Sec. 5.1.1)."""
    for row in read_golden_rows("table2_datasets.txt"):
        _, d, x = row[0], int(row[1]), int(row[2])
        assert oracle.default_x(d) == x, (d, x)


def _argmax_vertex_count(d):
    best, arg = -1, None
    for x in range(1, d + 1):
        c = math.comb(d, x) << x
        if c > best:  # strict: the smallest maximiser wins
            best, arg = c, x
    return arg


@pytest.mark.parametrize("d", list(range(1, 130)) + [200, 383, 384, 499, 500, 501, 768, 1000, 1024])
def test_default_x_is_smallest_maximiser_exact(d):
    assert oracle.default_x(d) == _argmax_vertex_count(d)


def test_vertex_count_powers_printed():
    """Table 2 prints the vertex count C(d,x)*2^x as a power of ten."""
    for row in read_golden_rows("table2_datasets.txt"):
        if row[3] == "-":
            continue
        d, x, p = int(row[1]), int(row[2]), int(row[3])
        count = math.comb(d, x) << x
        log10 = math.log10(count)
        # the table mixes truncation (10^46 for 10^46.64) and rounding
        # (10^182 for 10^181.85): accept either
        assert p in (math.floor(log10), round(log10)), (row, log10)


# ---------------------------------------------------------------- EVP set


def _vertices(d, x):
    """All {x,d} vertices (Sec. 2.3): d-vectors over {-1,0,1}, exactly x non-zeros."""
    out = []
    for pos in itertools.combinations(range(d), x):
        for signs in itertools.product((-1, 1), repeat=x):
            v = [0] * d
            for p, s in zip(pos, signs):
                v[p] = s
            out.append(v)
    return np.array(out, dtype=np.int8)


def test_cuboctahedron_vertices():
    """Figure 2: the {2,3} EVP is the cuboctahedron with 12 listed vertices."""
    printed = {tuple(int(v) for v in r) for r in read_golden_rows("fig2_cuboctahedron.txt")}
    assert len(printed) == 12
    enumerated = {tuple(int(v) for v in r) for r in _vertices(3, 2)}
    assert enumerated == printed
    # each vertex is its own nearest vertex
    V = np.array(sorted(printed), dtype=np.float32)
    assert {tuple(r) for r in oracle.encode(V, 2)} == printed


@pytest.mark.parametrize("d,x", [(3, 2), (5, 1), (6, 2), (8, 3), (7, 7)])
def test_vertex_count_formula(d, x):
    assert len(_vertices(d, x)) == math.comb(d, x) * 2 ** x


# ---------------------------------------------------------------- encoding


def test_worked_example_table3():
    g = read_golden("table3_worked_example.txt")
    x = int(g["x"][0])
    u1, u2 = _floats(g["u1"]), _floats(g["u2"])
    v1 = oracle.encode(u1[None], x)[0]
    v2 = oracle.encode(u2[None], x)[0]
    np.testing.assert_array_equal(v1, _ints(g["v1_printed"]))
    np.testing.assert_array_equal(v2, _ints(g["v2_rule"]))
    # the printed v2 is what the rule gives once u2[8] is negative
    u2_flip = u2.copy()
    u2_flip[8] = -u2_flip[8]
    np.testing.assert_array_equal(oracle.encode(u2_flip[None], x)[0], _ints(g["v2_printed"]))
    # bitplanes as printed
    T1 = oracle.pack(v1[None])[0]
    T2p = oracle.pack(_ints(g["v2_printed"])[None])[0]

    def bits(word):
        return [(int(word) >> j) & 1 for j in range(10)]

    assert bits(T1[0]) == [int(b) for b in g["v1plus_printed"]]
    assert bits(T1[1]) == [int(b) for b in g["v1minus_printed"]]
    assert bits(T2p[0]) == [int(b) for b in g["v2plus_printed"]]
    assert bits(T2p[1]) == [int(b) for b in g["v2minus_printed"]]
    # b2sp and Delta, for both readings of v2
    for v2x in (v2, _ints(g["v2_printed"])):
        assert oracle.dot(v1, v2x) == int(g["b2sp_v1_v2"][0])
        assert oracle.delta(v1, v2x) == int(g["delta_v1_v2"][0])


@pytest.mark.parametrize("d,x", [(6, 2), (8, 3), (5, 5), (7, 1), (6, 4)])
def test_encode_is_nearest_vertex_bruteforce(d, x):
    """Sec. 2.4: the encoding is the vertex maximising <u, v>, i.e. the nearest
    vertex on the hypersphere.  Checked against enumeration of all vertices."""
    V = _vertices(d, x).astype(np.float64)
    U = synth.uniform_sphere(10_000, d, stream=40 + d * 10 + x)
    scores = U.astype(np.float64) @ V.T
    top2 = np.sort(scores, axis=1)[:, -2:]
    assert np.all(top2[:, 1] - top2[:, 0] > 1e-12)  # unique nearest vertex
    best = V[np.argmax(scores, axis=1)].astype(np.int8)
    np.testing.assert_array_equal(oracle.encode(U, x), best)


def _check_code_invariants(U, V, x):
    n, d = U.shape
    nz = V != 0
    assert np.all(nz.sum(axis=1) == x)                       # exactly x non-zeros
    assert np.all((V.astype(np.int64) ** 2).sum(axis=1) == x)  # norm sqrt(x)
    assert np.all(np.isin(V, (-1, 0, 1)))
    # signs follow u for the selected elements
    assert np.all(V[nz] == np.where(U[nz] < 0, -1, 1))
    # every selected magnitude >= every unselected magnitude
    A = np.abs(U)
    sel_min = np.where(nz, A, np.inf).min(axis=1)
    uns_max = np.where(~nz, A, -np.inf).max(axis=1)
    assert np.all(sel_min >= uns_max)


@pytest.mark.parametrize("d,x,anis", [(384, 128, False), (100, 67, False), (768, 64, True),
                                      (65, 30, True), (63, 1, False), (64, 64, False)])
def test_encode_invariants_and_bitplanes(d, x, anis):
    U = synth.mixture_numpy(500, d, n_centres=16, anisotropic=anis, stream=7)
    V = oracle.encode(U, x)
    _check_code_invariants(U, V, x)
    T = oracle.pack(V)
    W = oracle.words(d)
    assert T.shape == (500, 2 * W)
    assert np.all(T[:, :W] & T[:, W:] == 0)                 # v+ and v- disjoint
    # set bits per row = x, and no bit beyond d
    popc = np.vectorize(lambda w: bin(int(w)).count("1"))
    assert np.all(popc(T).sum(axis=1) == x)
    if d % 64:
        pad = ~np.uint64((1 << (d % 64)) - 1)
        assert np.all(T[:, W - 1] & pad == 0) and np.all(T[:, 2 * W - 1] & pad == 0)
    V2, bad = oracle.unpack(T, d)
    assert bad == 0
    np.testing.assert_array_equal(V2, V)


def test_unpack_flags_malformed_rows():
    T = np.zeros((3, 2), dtype=np.uint64)
    T[0, 0] = 1; T[0, 1] = 1           # same dimension in both planes
    T[1, 0] = np.uint64(1) << np.uint64(40)   # bit beyond d = 10
    _, bad = oracle.unpack(T, 10)
    assert bad == 2


def test_encode_x_equals_d_is_sign_code():
    """Sec. 4.2: 1-bit quantisation is the {d,d} EVP -- every element keeps its sign."""
    U = synth.mixture_numpy(200, 96, stream=8)
    V = oracle.encode(U, 96)
    np.testing.assert_array_equal(V, np.where(U < 0, -1, 1).astype(np.int8))


def test_encode_permutation_equivariance():
    U = synth.uniform_sphere(300, 50, stream=9)
    assert all(len(set(np.abs(r).tolist())) == 50 for r in U)   # no magnitude ties
    perm = np.random.default_rng(3).permutation(50)
    np.testing.assert_array_equal(oracle.encode(U[:, perm], 20), oracle.encode(U, 20)[:, perm])


def test_encode_power_of_two_scale_invariance():
    U = synth.mixture_numpy(300, 128, stream=10)
    V = oracle.encode(U, 85)
    for s in (0.125, 32.0):
        np.testing.assert_array_equal(oracle.encode(U * np.float32(s), 85), V)


def test_encode_tie_and_zero_readings():
    # equal magnitudes: lower index first; a selected -0.0 or +0.0 is +1
    u = np.array([[0.5, -0.5, 0.5, -0.5, 0.25]], dtype=np.float32)
    np.testing.assert_array_equal(oracle.encode(u, 3)[0], [1, -1, 1, 0, 0])
    z = np.array([[0.0, -0.0, 0.0, 0.3]], dtype=np.float32)
    np.testing.assert_array_equal(oracle.encode(z, 3)[0], [1, 1, 0, 1])


def test_encode_rejects_nonfinite():
    u = np.array([[0.1, np.nan, 0.2]], dtype=np.float32)
    with pytest.raises(oracle.NonFiniteInput):
        oracle.encode(u, 2)
    u = np.array([[0.1, np.inf, 0.2]], dtype=np.float32)
    with pytest.raises(oracle.NonFiniteInput):
        oracle.encode(u, 2)


# ---------------------------------------------------------------- b2sp / Delta


def _b2sp_from_bitplanes(t1, t2, W):
    """The paper's four-term definition (Sec. 5.1.2):
    b2sp = bsp(v+,w+) + bsp(v-,w-) - bsp(v+,w-) - bsp(v-,w+), bsp = popcount(v & w)."""
    def bsp(a, b):
        return sum(bin(int(a[i]) & int(b[i])).count("1") for i in range(W))
    vp, vm, wp, wm = t1[:W], t1[W:], t2[:W], t2[W:]
    return bsp(vp, wp) + bsp(vm, wm) - bsp(vp, wm) - bsp(vm, wp)


@pytest.mark.parametrize("d,x", [(10, 5), (64, 40), (100, 67), (130, 7), (384, 256)])
def test_dot_equals_four_term_b2sp(d, x):
    V = synth.ternary_random(40, d, x, stream=11)
    T = oracle.pack(V)
    W = oracle.words(d)
    for i in range(0, 40, 2):
        assert oracle.dot(V[i], V[i + 1]) == _b2sp_from_bitplanes(T[i], T[i + 1], W)


@pytest.mark.parametrize("d,x", [(10, 5), (100, 67), (384, 128)])
def test_delta_properties(d, x):
    V = synth.ternary_random(60, d, x, stream=12)
    for i in range(0, 57, 3):
        a, b, c = V[i], V[i + 1], V[i + 2]
        dab = oracle.delta(a, b)
        assert oracle.delta(a, a) == 0
        assert dab == oracle.delta(b, a)
        assert dab % 2 == 0 and 0 <= dab <= 4 * x
        assert dab == 2 * x - 2 * oracle.dot(a, b)          # closed form for equal-x codes
        # sqrt(Delta) is a Euclidean distance: triangle inequality
        assert math.sqrt(dab) <= math.sqrt(oracle.delta(a, c)) + math.sqrt(oracle.delta(c, b)) + 1e-12
    # extremes: identical code -> 0, negated code -> 4x
    assert oracle.delta(V[0], -V[0]) == 4 * x


# ---------------------------------------------------------------- kNN


def _knn_python(Vq, Vs, k):
    out_ids, out_d = [], []
    for q in Vq:
        ql = [int(t) for t in q]
        keys = []
        for s_idx, s in enumerate(Vs):
            dd = sum((a - int(b)) ** 2 for a, b in zip(ql, s))
            keys.append((dd, s_idx))
        keys.sort()
        out_ids.append([i for _, i in keys[:k]])
        out_d.append([dd for dd, _ in keys[:k]])
    return np.array(out_ids), np.array(out_d)


def test_knn_bruteforce_with_ties():
    Vs = synth.ternary_random(60, 16, 5, stream=13)
    Vs[30] = Vs[3]
    Vs[45] = Vs[3]            # equal distances for every query: tie-break by index
    Vq = np.concatenate([synth.ternary_random(6, 16, 5, stream=14), Vs[3:4]])
    for k in (1, 7, 60):
        ids, dist = oracle.knn(Vq, Vs, k)
        pids, pd = _knn_python(Vq, Vs, k)
        np.testing.assert_array_equal(ids, pids)
        np.testing.assert_array_equal(dist, pd)
    ids, dist = oracle.knn(Vs[3:4], Vs, 3)
    assert ids[0].tolist() == [3, 30, 45] and dist[0].tolist() == [0, 0, 0]


def test_knn_shard_merge_invariance():
    U = synth.mixture_numpy(3000, 64, stream=15)
    Q = synth.mixture_numpy(20, 64, stream=16)
    Vs, Vq = oracle.encode(U, 43), oracle.encode(Q, 43)
    k = 25
    ids, dist = oracle.knn(Vq, Vs, k)
    bounds = [0, 700, 1900, 3000]
    parts_i, parts_d = [], []
    for a, b in zip(bounds[:-1], bounds[1:]):
        i, dd = oracle.knn(Vq, Vs[a:b], k)
        parts_i.append(i + a)
        parts_d.append(dd)
    I = np.concatenate(parts_i, axis=1)
    D = np.concatenate(parts_d, axis=1)
    for q in range(len(Vq)):
        order = np.lexsort((I[q], D[q]))[:k]
        np.testing.assert_array_equal(I[q][order], ids[q])
        np.testing.assert_array_equal(D[q][order], dist[q])


def test_knn_argument_checks():
    V = synth.ternary_random(5, 8, 3, stream=17)
    with pytest.raises(ValueError):
        oracle.knn(V, V, 6)
    with pytest.raises(ValueError):
        oracle.knn(V, V, 0)


# ---------------------------------------------------------------- rerank


def test_rerank_closed_form_and_ties():
    d = 4
    S = np.array([[1, 0, 0, 0], [0.5, 0.5, 0, 0], [0, 1, 0, 0],
                  [0.5, 0.5, 0, 0], [-1, 0, 0, 0]], dtype=np.float32)
    Q = np.array([[1, 0, 0, 0], [0, 0, 0, 1]], dtype=np.float32)
    sl = np.array([[4, 3, 1, 0, -1, 2], [0, 1, 2, 3, 4, -1]], dtype=np.int64)
    ids, sc, ab = oracle.rerank(Q, S, sl, 4)
    assert ids[0].tolist() == [0, 1, 3, 2]          # 1.0, 0.5 (idx 1 before 3), 0.0
    assert sc[0].tolist() == [1.0, 0.5, 0.5, 0.0]
    assert ids[1].tolist() == [0, 1, 2, 3]          # all scores 0: index order
    assert sc[1].tolist() == [0.0] * 4
    # fewer valid entries than k -> -1 / -inf tail
    ids, sc, _ = oracle.rerank(Q[:1], S, np.array([[2, -1, -1]]), 3)
    assert ids[0].tolist() == [2, -1, -1] and sc[0, 1] == -np.inf
    with pytest.raises(ValueError):
        oracle.rerank(Q[:1], S, np.array([[5]]), 1)


def test_rerank_matches_float64_matmul():
    S = synth.mixture_numpy(2000, 96, stream=18)
    Q = synth.mixture_numpy(10, 96, stream=19)
    rng = np.random.default_rng(4)
    sl = np.stack([rng.choice(2000, 50, replace=False) for _ in range(10)])
    ids, sc, ab = oracle.rerank(Q, S, sl, 10)
    full = Q.astype(np.float64) @ S.astype(np.float64).T
    for q in range(10):
        cand = sl[q]
        order = sorted(cand.tolist(), key=lambda i: (-full[q, i], i))[:10]
        assert ids[q].tolist() == order
        np.testing.assert_allclose(sc[q], full[q, ids[q]], rtol=0, atol=1e-12)
        np.testing.assert_allclose(ab[q], np.abs(Q[q].astype(np.float64) * S[ids[q]].astype(np.float64)).sum(1),
                                   rtol=1e-12)


# ---------------------------------------------------------------- statistics


def _spearman(a, b):
    from scipy.stats import spearmanr
    return spearmanr(a, b).correlation


def _b158(U):
    """BitNet b1.58 ternarisation (Sec. 4.3), gamma taken per vector (reading)."""
    gamma = np.mean(np.abs(U), axis=1, keepdims=True)
    return np.clip(np.rint(U / (gamma + 1e-8)), -1, 1)


@pytest.mark.parametrize("d,rho_paper", [(100, 0.80), (1000, 0.79)])
def test_spearman_uniform_rows_of_table2(d, rho_paper):
    """Table 2, 'Uniform' rows: EVP correlates best, b1.58 next, 1-bit last, and
    the EVP correlation is close to the printed value (sampled pairs; the
    paper does not state its sampling, so a 0.05 band is allowed)."""
    n, pairs = 2000, 20000
    U = synth.uniform_sphere(n, d, stream=20 + d)
    rng = np.random.default_rng(5)
    i = rng.integers(0, n, pairs)
    j = rng.integers(0, n, pairs)
    keep = i != j
    i, j = i[keep], j[keep]
    true = np.linalg.norm(U[i].astype(np.float64) - U[j], axis=1)
    x = oracle.default_x(d)
    E = oracle.encode(U, x).astype(np.int64)
    B1 = oracle.encode(U, d).astype(np.int64)       # 1-bit = {d,d} EVP
    BT = _b158(U.astype(np.float64))
    evp = ((E[i] - E[j]) ** 2).sum(1)
    one = ((B1[i] - B1[j]) ** 2).sum(1)
    b158 = ((BT[i] - BT[j]) ** 2).sum(1)
    r_evp, r_one, r_b = _spearman(true, evp), _spearman(true, one), _spearman(true, b158)
    assert r_evp > r_b > r_one
    assert abs(r_evp - rho_paper) < 0.05, r_evp


def test_equal_volume_selection_frequencies():
    """Sec. 2.5: for uniform points every vertex is equally likely, so each
    coordinate is selected with frequency x/d and signs split evenly."""
    d, x, n = 30, 20, 20000
    V = oracle.encode(synth.uniform_sphere(n, d, stream=21), x)
    freq = (V != 0).mean(axis=0)
    sd = math.sqrt((x / d) * (1 - x / d) / n)
    assert np.all(np.abs(freq - x / d) < 5 * sd)
    pos = (V == 1).sum(axis=0) / (V != 0).sum(axis=0)
    assert np.all(np.abs(pos - 0.5) < 5 * math.sqrt(0.25 / (n * x / d)))
