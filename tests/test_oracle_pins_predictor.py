"""Pins of the oracle's disparity predictor g_psi (CPU only): the level
resolutions' geometric progression, the hash index's structure (a bijection
in the dense regime; xor-separable with pi_1 = 1 in the hashed one), exact
reproduction of a linear field by the trilinear encoding, and a hand-built
MLP whose output is exp(omega_r . e_z)."""
import numpy as np
import pytest

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I


def test_resolutions():
    r = O.hash_resolutions(8, 16, 512)
    assert r[0] == 16 and r[-1] == 512
    ratios = [b / a for a, b in zip(r[:-1], r[1:])]
    assert all(1.5 < q < 1.75 for q in ratios)        # b = 32^(1/7) = 1.64, floored
    assert O.hash_resolutions(1, 16, 512) == [16]


def test_hash_index_structure():
    # dense: every vertex of a 9^3 grid gets its own entry in [0, 729)
    g = np.stack(np.meshgrid(np.arange(9), np.arange(9), np.arange(9), indexing="ij"), -1).reshape(-1, 3)
    d = O.hash_index(g[:, 0], g[:, 1], g[:, 2], 8, 4096)
    assert sorted(d.tolist()) == list(range(729))
    # hashed (40^3 > T): the first prime is 1 and the hash xor-separates
    T = 1 << 12
    rng = np.random.default_rng(1)
    i, j, k = (rng.integers(0, 40, 500) for _ in range(3))
    h = O.hash_index(i, j, k, 39, T)
    z = np.zeros_like(i)
    assert np.all(O.hash_index(i, z, z, 39, T) == i % T)
    assert np.all(h == O.hash_index(i, z, z, 39, T) ^ O.hash_index(z, j, z, 39, T)
                  ^ O.hash_index(z, z, k, 39, T))
    assert np.all((h >= 0) & (h < T)) and O.hash_index(0, 0, 0, 39, T) == 0
    assert len(np.unique(h)) > 400                     # the primes spread the vertices


@pytest.mark.parametrize("x_edge", [False, True])
def test_encoding_reproduces_a_linear_field(x_edge):
    """Dense levels whose entries hold a linear function of the vertex
    coordinates: the trilinear blend returns that function at p = x N_l."""
    res = [4, 7, 13]
    T = 14 ** 3
    F = 2
    coef = np.array([[0.5, -1.0, 2.0, 0.25], [1.5, 0.75, -0.5, -1.0]])
    table = np.zeros((len(res), T, F))
    for l, N in enumerate(res):
        g = np.stack(np.meshgrid(np.arange(N + 1), np.arange(N + 1), np.arange(N + 1),
                                 indexing="ij"), -1).reshape(-1, 3)
        idx = O.hash_index(g[:, 0], g[:, 1], g[:, 2], N, T)
        for f in range(F):
            table[l, idx, f] = g @ coef[f, :3] + coef[f, 3] * (l + 1)
    x = I.rng(3).random((300, 3)).astype(np.float32)
    if x_edge:
        x[:50] = np.float32(1.0)
        x[50:100, 0] = np.float32(0.0)
    enc = O.hash_encode(table, res, x)
    for l, N in enumerate(res):
        p = (x * np.float32(N)).astype(np.float64)
        for f in range(F):
            want = p @ coef[f, :3] + coef[f, 3] * (l + 1)
            np.testing.assert_allclose(enc[:, l * F + f], want, rtol=1e-12, atol=1e-12)


def test_predictor_hand_mlp():
    """W1 routes omega_r's z component into two ReLU units (+z, -z), W2 is
    the identity, W3 = (1, -1): z = omega_r . e_z and d = exp(z)."""
    res = [4, 8]
    table = I.rng(4).normal(size=(2, 64, 2))
    W1 = np.zeros((2, 2 * 2 + 3))
    W1[0, 6], W1[1, 6] = 1.0, -1.0
    W2 = np.eye(2)
    W3 = np.array([[1.0, -1.0]])
    g = I.rng(5)
    x = g.random((200, 3)).astype(np.float32)
    w = I.unit_vectors(g, 200).astype(np.float32)
    n = I.unit_vectors(g, 200).astype(np.float32)
    d = O.disparity(table, res, [W1, W2, W3], x, w, n)
    r = O.reflect_f32(w, n).astype(np.float64)
    np.testing.assert_allclose(d, np.exp(r[:, 2]), rtol=1e-14)


def test_decoder_attributes():
    """Eq. 12: attributes behind zero columns of W1 change nothing; with an
    all-zero table the hand decoder returns exp(g_0) in the first channel."""
    ot = O.build_tree(61, 2, 1.0, [4, 4, 4])
    g = I.rng(62)
    x = g.random((100, 3)).astype(np.float32)
    w = I.unit_vectors(g, 100).astype(np.float32)
    tables = I.make_tables(63, ot.num_texels, 4, 0.5)
    W = I.make_mlp(64, [12, 16, 16, 3])
    attrs = g.normal(size=(100, 13))
    W1z = np.concatenate([W[0], np.zeros((16, 13))], axis=1)
    a, _ = O.query_forward(ot, tables, [W1z, W[1], W[2]], x, w, attrs=attrs)
    b, _ = O.query_forward(ot, tables, W, x, w)
    np.testing.assert_array_equal(a, b)
    W1 = np.zeros((2, 25))
    W1[0, 12], W1[1, 12] = 1.0, -1.0
    W3 = np.zeros((3, 2))
    W3[0] = [1.0, -1.0]
    rgb, _ = O.query_forward(ot, np.zeros_like(tables), [W1, np.eye(2), W3], x, w, attrs=attrs)
    np.testing.assert_allclose(rgb[:, 0], np.exp(attrs[:, 0]), rtol=1e-15)
    np.testing.assert_array_equal(rgb[:, 1:], 1.0)


def test_shifted_features_derivative_in_d():
    """dh/dd of the shifted lookup against central differences in d (step
    1e-3 d, queries whose binary32 decisions change across the step left
    out; the binary32 fractions bound the differences' accuracy to ~1e-3)."""
    ot = O.build_tree(81, 3, 0.8, [17, 9, 9, 5])
    tables = I.make_tables(82, ot.num_texels, 4, 0.5)
    g = I.rng(83)
    n = 300
    x = g.random((n, 3)).astype(np.float32)
    w = I.unit_vectors(g, n).astype(np.float32)
    nrm = I.unit_vectors(g, n).astype(np.float32)
    d = g.uniform(0.5, 4.0, n).astype(np.float32)
    an = O.shifted_features_d_gradient(ot, tables, x, w, nrm, d)
    dp = (d * np.float32(1.001)).astype(np.float32)
    dm = (d * np.float32(0.999)).astype(np.float32)
    ep = O.encode_features_shifted(ot, tables, x, w, nrm, dp)
    em = O.encode_features_shifted(ot, tables, x, w, nrm, dm)
    e0 = O.encode_features_shifted(ot, tables, x, w, nrm, d)
    same = np.all((ep.addr == e0.addr) & (em.addr == e0.addr), axis=(1, 2, 3))
    assert same.sum() > n // 3
    fd = (ep.h - em.h) / (dp.astype(np.float64) - dm.astype(np.float64))[:, None]
    a, f = an[same], fd[same]
    assert np.linalg.norm(a - f) <= 3e-3 * np.linalg.norm(f)
    assert np.linalg.norm(f) > 0


def test_predictor_backward_by_central_differences():
    """g_psi's table and weight gradients of sum_q c_q d_q against central
    differences (FP64; the encoding is linear in the table)."""
    table, res = None, [4, 9]
    rng = np.random.default_rng(84)
    table = rng.uniform(-0.3, 0.3, (2, 64, 2))
    weights = [W.astype(np.float64) * 1.5 for W in I.make_mlp(85, [7, 16, 16, 1])]
    g = I.rng(86)
    n = 50
    x = g.random((n, 3)).astype(np.float32)
    w = I.unit_vectors(g, n).astype(np.float32)
    nrm = I.unit_vectors(g, n).astype(np.float32)
    c = rng.normal(size=n)

    def f(tab, Ws):
        return float(np.sum(c * O.disparity(tab, res, Ws, x, w, nrm)))
    dtab, dWs = O.disparity_backward(table, res, weights, x, w, nrm, c)
    h = 1e-6
    touched = np.argwhere(np.abs(dtab) > 0)
    for (l, e, k) in touched[rng.choice(len(touched), 12, replace=False)]:
        P, Q = table.copy(), table.copy()
        P[l, e, k] += h
        Q[l, e, k] -= h
        assert dtab[l, e, k] == pytest.approx((f(P, weights) - f(Q, weights)) / (2 * h), rel=1e-5,
                                              abs=1e-9)
    for i in range(3):
        a, b = int(rng.integers(weights[i].shape[0])), int(rng.integers(weights[i].shape[1]))
        P = [W.copy() for W in weights]
        Q = [W.copy() for W in weights]
        P[i][a, b] += h
        Q[i][a, b] -= h
        assert dWs[i][a, b] == pytest.approx((f(table, P) - f(table, Q)) / (2 * h), rel=1e-5,
                                             abs=1e-9)


def test_hash_index_published_primes_worked_examples():
    """The spatial hash against index values worked out by hand from the
    published primes (tests/golden/hash_index_mueller2022.txt): a wrong
    pi_2 or pi_3, or a sum in place of the xor, fails it."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "hash_index_mueller2022.txt")
    rows = [list(map(int, ln.split())) for ln in open(path)
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 5
    for i, j, k, res, T, want in rows:
        assert int(O.hash_index(i, j, k, res, T)) == want, (i, j, k, res, T)
