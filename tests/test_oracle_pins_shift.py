"""Pins of the oracle's disparity-shifted lookup (Eq. 7-9; CPU only): the
reflection against closed forms and its invariants, the shifted direction
against Eq. 8's virtual point y = x + omega_r / d in FP64, the zero-disparity
case against the unshifted full form (pinned on its own), and every cell's
vertex entries against a brute-force per-cell lookup."""
import numpy as np
import pytest

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I


def test_reflection_closed_forms_and_invariants():
    s = np.float32(1 / np.sqrt(2))
    w = np.array([[s, 0, s], [0, 0, 1], [1, 0, 0], [0.6, 0.0, 0.8]], np.float32)
    n = np.array([[0, 0, 1], [0, 0, 1], [0, 0, 1], [0, 0, 1]], np.float32)
    r = O.reflect_f32(w, n)
    np.testing.assert_allclose(r, [[-s, 0, s], [0, 0, 1], [-1, 0, 0], [-0.6, 0, 0.8]], atol=1e-7)
    g = I.rng(5)
    w = I.unit_vectors(g, 500)
    n = I.unit_vectors(g, 500)
    r = O.reflect_f32(w * 3.0, n * 0.5).astype(np.float64)  # lengths are normalised away
    np.testing.assert_allclose(np.linalg.norm(r, axis=1), 1.0, atol=1e-6)
    np.testing.assert_allclose(np.sum(r * n, 1), np.sum(w * n, 1), atol=1e-6)   # same angle to n
    np.testing.assert_allclose(r + w, 2 * np.sum(w * n, 1)[:, None] * n, atol=1e-6)  # in the plane of n, w
    np.testing.assert_allclose(O.reflect_f32(r, n), w, atol=2e-6)                 # an involution


def test_shifted_direction_points_from_the_cell_centre_to_eq8_point():
    """v = (x - c) d + omega_r is parallel to y - c with y = x + omega_r / d
    (Eq. 8), for every cell of the eight around x."""
    g = I.rng(6)
    x = g.random((400, 3)).astype(np.float32)
    om_r = I.unit_vectors(g, 400).astype(np.float32)
    d = g.uniform(0.05, 20.0, 400).astype(np.float32)
    for l in (0, 2, 5):
        cells, _, _ = O.neighbour_cells(x, l)
        for j in range(8):
            v = O.shifted_direction_f32(x, om_r, d, cells[:, j], l).astype(np.float64)
            c = (cells[:, j] + 0.5) / 2.0 ** l
            y = x.astype(np.float64) + om_r.astype(np.float64) / d[:, None]
            u = y - c
            cos = np.sum(u * v, 1) / (np.linalg.norm(u, axis=1) * np.linalg.norm(v, axis=1))
            assert np.all(cos > 1 - 1e-9), (l, j, cos.min())


def _tree_and_tables(seed, depth, V, F=4):
    ot = O.build_tree(seed, depth, 1.0 if depth <= 2 else 0.6, V)
    tables = I.make_tables(seed + 1, ot.num_texels, F, 0.5)
    return ot, tables


def test_zero_disparity_is_the_full_form_at_the_reflection():
    ot, tables = _tree_and_tables(41, 4, [9, 9, 5, 5, 3])
    g = I.rng(42)
    x = g.random((700, 3)).astype(np.float32)
    w = I.unit_vectors(g, 700).astype(np.float32)
    n = I.unit_vectors(g, 700).astype(np.float32)
    a = O.encode_features_shifted(ot, tables, x, w, n, np.zeros(700, np.float32))
    b = O.encode_features_full(ot, tables, x, O.reflect_f32(w, n))
    np.testing.assert_array_equal(a.addr, b.addr)
    np.testing.assert_array_equal(a.weight, b.weight)
    np.testing.assert_allclose(a.h, b.h, rtol=1e-12, atol=1e-15)   # summation order differs


def test_each_cell_looks_up_its_own_direction():
    """Brute force per cell: the direction of y - c_j from Eq. 8 in FP64,
    rounded to binary32, its vertex cell and triangle on the node's map;
    the oracle's entries agree wherever the binary32 decisions are more than
    1e-4 from a cell or triangle boundary, and at d > 0 the cells' entries
    differ from the unshifted form's."""
    V = [9, 9, 5, 5]
    ot, tables = _tree_and_tables(51, 3, V)
    g = I.rng(52)
    n_q = 300
    x = g.random((n_q, 3)).astype(np.float32)
    w = I.unit_vectors(g, n_q).astype(np.float32)
    nrm = I.unit_vectors(g, n_q).astype(np.float32)
    d = g.uniform(0.5, 8.0, n_q).astype(np.float32)
    enc = O.encode_features_shifted(ot, tables, x, w, nrm, d)
    om_r = O.reflect_f32(w, nrm).astype(np.float64)
    y = x.astype(np.float64) + om_r / d[:, None].astype(np.float64)
    checked = 0
    for l in range(ot.num_levels):
        Vl = V[l]
        N = Vl - 1
        cells, _, _ = O.neighbour_cells(x, l)
        for j in range(8):
            u = (y - (cells[:, j] + 0.5) / 2.0 ** l).astype(np.float32)
            i0, j0, fx, fy = O.vertex_cell_f32(u, Vl)
            off, _ = O.vertex_triangle(i0, j0, fx, fy, N)
            safe = (np.minimum.reduce([fx, 1 - fx, fy, 1 - fy, np.abs(fx + fy - 1),
                                       np.abs(fx - fy)]) > 1e-4)
            for k in range(3):
                vi, vj = O.canonical_vertex(i0 + off[:, k, 0], j0 + off[:, k, 1], N)
                a = enc.addr[:, l, j, k]
                present = a >= 0
                base = a - (vj * Vl + vi)
                ok = safe & present
                # the entry lies in the cell's own map: the same base for the three vertices
                assert np.all(base[ok] == np.asarray(ot.map_offset)[np.maximum(
                    O.node_of_cell(ot, l, np.clip(cells[ok, j], 0, None)), 0)])
                checked += int(ok.sum())
    assert checked > 2000
    full = O.encode_features_full(ot, tables, x, O.reflect_f32(w, nrm))
    assert np.mean(enc.addr != full.addr) > 0.1


def test_shifted_backward_by_central_differences():
    """Table and weight gradients of sum(d_rgb . L_hat) in the shifted form
    against central differences of the forward (the disparity fixed; step
    1e-6, so the differences carry ~1e-6 relative rounding of sum's size)."""
    ot, tables = _tree_and_tables(71, 2, [5, 5, 3])
    g = I.rng(72)
    n = 40
    x = g.random((n, 3)).astype(np.float32)
    w = I.unit_vectors(g, n).astype(np.float32)
    nrm = I.unit_vectors(g, n).astype(np.float32)
    d = g.uniform(0.5, 5.0, n).astype(np.float32)
    weights = [W.astype(np.float64) * 2 for W in I.make_mlp(73, [12, 16, 16, 3])]
    d_rgb = g.normal(size=(n, 3))
    T = tables.astype(np.float64)

    def f(T_, Ws_):
        rgb, _ = O.query_forward(ot, T_, Ws_, x, w, form="shifted", normal=nrm, disparity=d)
        return float(np.sum(d_rgb * rgb))
    dT, dWs, _ = O.query_backward(ot, T, weights, x, w, d_rgb, form="shifted", normal=nrm,
                                  disparity=d)
    h = 1e-6
    touched = np.nonzero(np.abs(dT).sum(1) > 0)[0]
    for r in g.choice(touched, 10, replace=False):
        c = int(g.integers(4))
        P, Q = T.copy(), T.copy()
        P[r, c] += h
        Q[r, c] -= h
        assert dT[r, c] == pytest.approx((f(P, weights) - f(Q, weights)) / (2 * h), rel=1e-5,
                                         abs=1e-8)
    for i in range(3):
        a, b = int(g.integers(weights[i].shape[0])), int(g.integers(weights[i].shape[1]))
        P = [W.copy() for W in weights]
        Q = [W.copy() for W in weights]
        P[i][a, b] += h
        Q[i][a, b] -= h
        assert dWs[i][a, b] == pytest.approx((f(T, P) - f(T, Q)) / (2 * h), rel=1e-5, abs=1e-8)
