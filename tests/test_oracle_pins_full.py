"""Pins of the oracle's full query form (Eq. 6 barycentric interpolation on
vertex maps, Eq. 10 eight-cell renormalised trilinear blend) against closed
forms, brute force and invariants, independent of the oracle's own code
paths."""
import numpy as np
import pytest

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I


def _uv(omega):
    return O.octa_uv(np.asarray(omega, np.float32).astype(np.float64))


def test_node_of_cell_matches_bruteforce():
    t = O.build_tree(11, 4, 0.7, [3, 3, 3, 3, 3])
    rng = np.random.default_rng(0)
    for l in range(5):
        c = rng.integers(0, 1 << l, size=(400, 3))
        np.testing.assert_array_equal(O.node_of_cell(t, l, c), O.node_of_cell_bruteforce(t, l, c))


def test_trilinear_weights_closed_form():
    x = np.random.default_rng(1).random((500, 3)).astype(np.float32)
    for l in (0, 1, 3, 5):
        cells, w, inside = O.neighbour_cells(x, l)
        np.testing.assert_allclose(w.sum(1), 1.0, atol=1e-12)
        # the weighted cell centres reproduce x (linear precision)
        centres = (cells + 0.5) / (1 << l)
        np.testing.assert_allclose((w[:, :, None] * centres).sum(1), x.astype(np.float64), atol=1e-12)
        assert np.all(w >= -1e-12)
    # x at a cell centre: all weight on that cell
    c = np.array([[3, 5, 6]])
    xc = ((c + 0.5) / 8).astype(np.float32)
    cells, w, _ = O.neighbour_cells(xc, 3)
    j = int(np.argmax(w[0]))
    assert w[0, j] == pytest.approx(1.0) and np.all(cells[0, j] == c[0])


def _directions(n, seed):
    _, w = I.uniform_queries(seed, n)
    return w


@pytest.mark.parametrize("V", [3, 5, 9, 33])
def test_barycentric_reconstructs_the_point_inside_one_face(V):
    N = V - 1
    w = _directions(3000, V)
    i0, j0, fx, fy = O.vertex_cell_f32(w, V)
    off, b = O.vertex_triangle(i0, j0, fx, fy, N)
    assert np.all(b >= -1e-6)
    np.testing.assert_allclose(b.sum(1), 1.0, atol=1e-12)
    vu = (i0[:, None] + off[:, :, 0]) / N
    vv = (j0[:, None] + off[:, :, 1]) / N
    uv = _uv(w)
    np.testing.assert_allclose((b * vu).sum(1), uv[:, 0], atol=1e-6)
    np.testing.assert_allclose((b * vv).sum(1), uv[:, 1], atol=1e-6)
    # the three vertices lie in one octahedron face: none strictly on the
    # other side of |u_x| + |u_y| = 1 from another
    d = np.abs(2 * vu - 1) + np.abs(2 * vv - 1) - 1
    assert not np.any((d.max(1) > 1e-12) & (d.min(1) < -1e-12))
    # and in one quadrant
    for a in (2 * vu - 1, 2 * vv - 1):
        assert not np.any((a.max(1) > 1e-12) & (a.min(1) < -1e-12))


@pytest.mark.parametrize("V", [3, 5, 17])
def test_identified_border_vertices_are_one_direction(V):
    N = V - 1
    ii, jj = np.meshgrid(np.arange(V), np.arange(V), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    ci, cj = O.canonical_vertex(ii, jj, N)
    u = np.stack([2 * ii / N - 1, 2 * jj / N - 1], 1)
    cu = np.stack([2 * ci / N - 1, 2 * cj / N - 1], 1)
    np.testing.assert_allclose(O.octa_decode(u), O.octa_decode(cu), atol=1e-12)
    ci2, cj2 = O.canonical_vertex(ci, cj, N)
    np.testing.assert_array_equal(ci2, ci)
    np.testing.assert_array_equal(cj2, cj)
    # distinct directions keep distinct representatives: an octahedron with
    # every edge cut in m = N / 2 has 4 m^2 + 2 = N^2 + 2 vertices
    reps = set(zip(ci.tolist(), cj.tolist()))
    assert len(reps) == N * N + 2


def test_constant_table_gives_the_constant_where_a_neighbour_exists():
    t = O.build_tree(21, 3, 0.6, [9, 9, 5, 3])
    x, w = I.uniform_queries(22, 2000)
    T = np.full((t.num_texels, 4), 0.37)
    e = O.encode_features_full(t, T, x, w)
    for l in range(t.num_levels):
        cells, _, inside = O.neighbour_cells(x, l)
        any_present = np.zeros(len(x), bool)
        for j in range(8):
            nd = O.node_of_cell_bruteforce(t, l, np.clip(cells[:, j], 0, (1 << l) - 1))
            any_present |= inside[:, j] & (nd >= 0)
        hl = e.h[:, 4 * l:4 * l + 4]
        np.testing.assert_allclose(hl[any_present], 0.37, atol=1e-12)
        assert np.all(hl[~any_present] == 0.0)


def test_level_without_a_present_neighbour_is_zero():
    """Only octant 0 of the root is split: a point near (1, 1, 1) has no
    level-2 cell around it, a point near the origin has all eight."""
    t = O.tree_from_flags([1, 1, 0, 0, 0, 0, 0, 0, 0], 2, [3, 3, 3])
    T = np.full((t.num_texels, 2), 1.5)
    x = np.array([[0.9, 0.9, 0.9], [0.2, 0.2, 0.2]], np.float32)
    w = np.array([[0.0, 0.0, 1.0], [0.3, -0.2, 0.9]], np.float32)
    e = O.encode_features_full(t, T, x, w)
    assert np.all(e.h[0, 4:6] == 0.0) and np.all(e.addr[0, 2] == -1)
    np.testing.assert_allclose(e.h[1, 4:6], 1.5, atol=1e-12)
    assert np.all(e.addr[1, 2] >= 0)


def test_trilinear_reproduces_a_linear_field_on_a_dense_tree():
    """Every entry of a node equal to a . centre(node) + b: where all eight
    cells exist, h_l(x) = a . x + b exactly."""
    t = O.build_tree(31, 3, 1.0, [3, 3, 3, 3])
    a, b0 = np.array([0.3, -1.1, 0.7]), 0.25
    T = np.zeros((t.num_texels, 1))
    for n in range(t.num_nodes):
        l = int(np.searchsorted(t.level_node_start, n, side="right") - 1)
        centre = (t.node_coord[n] + 0.5) / (1 << l)
        V = t.R[l]
        T[t.map_offset[n]:t.map_offset[n] + V * V, 0] = a @ centre + b0
    x, w = I.uniform_queries(32, 3000)
    e = O.encode_features_full(t, T, x, w)
    x64 = x.astype(np.float64)
    for l in range(t.num_levels):
        m = np.all((x64 > 0.5 / (1 << l)) & (x64 < 1 - 0.5 / (1 << l)), axis=1)
        np.testing.assert_allclose(e.h[m, l], x64[m] @ a + b0, atol=1e-9)


def test_barycentric_reproduces_a_linear_field_of_the_direction():
    """Root-only tree, vertex values linear in (u, v): upper-hemisphere
    directions away from the square's edge get the linear field itself."""
    V = 17
    t = O.tree_from_flags([], 0, [V])
    alpha, beta, gam = 0.8, -0.45, 0.1
    ii, jj = np.meshgrid(np.arange(V), np.arange(V), indexing="ij")
    T = np.zeros((V * V, 1))
    T[jj.ravel() * V + ii.ravel(), 0] = alpha * ii.ravel() / (V - 1) + beta * jj.ravel() / (V - 1) + gam
    w = _directions(4000, 40)
    w = w[w[:, 2] > 0.2]
    e = O.encode_features_full(t, T, np.full((len(w), 3), 0.5, np.float32), w)
    uv = _uv(w)
    np.testing.assert_allclose(e.h[:, 0], alpha * uv[:, 0] + beta * uv[:, 1] + gam, atol=1e-6)


def test_directional_features_are_continuous_on_the_sphere():
    """Random vertex values: directions an arc of 1e-6 apart, seams and face
    edges included, give features within a Lipschitz bound."""
    V = 9
    t = O.tree_from_flags([], 0, [V])
    T = np.random.default_rng(5).normal(size=(V * V, 2))
    rng = np.random.default_rng(6)
    w = _directions(3000, 41).astype(np.float64)
    # half of them pushed close to the lower hemisphere's fold edges
    near = w.copy()
    near[:, 2] = -np.abs(near[:, 2])
    near[:, 0] *= 1e-3
    w = np.concatenate([w, near])
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    d = rng.normal(size=w.shape)
    d -= (d * w).sum(1, keepdims=True) * w
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    w2 = w + 1e-6 * d
    x = np.full((len(w), 3), 0.5, np.float32)
    h1 = O.encode_features_full(t, T, x, w.astype(np.float32)).h
    h2 = O.encode_features_full(t, T, x, w2.astype(np.float32)).h
    lip = 4 * (V - 1) * np.abs(T).max() * 2
    assert np.max(np.abs(h1 - h2)) <= lip * 2e-6 + 1e-6


def test_full_form_backward_matches_central_differences():
    """d/dtheta of sum(d_rgb . L_hat) in the full form: the oracle's analytic
    table and weight gradients against central differences (FP64)."""
    t = O.build_tree(41, 2, 0.8, [5, 3, 3])
    F = 2
    rng = np.random.default_rng(42)
    T = rng.normal(scale=0.3, size=(t.num_texels, F))
    Ws = [W.astype(np.float64) * 1.5 for W in I.make_mlp(43, [t.num_levels * F, 8, 3])]
    x, w = I.uniform_queries(44, 40)
    d = rng.normal(size=(len(x), 3))
    dT, dWs, _ = O.query_backward(t, T, Ws, x, w, d, form="full")

    def f(T_, Ws_):
        rgb, _ = O.query_forward(t, T_, Ws_, x, w, form="full")
        return float(np.sum(d * rgb))

    h = 1e-6
    touched = np.argwhere(np.abs(dT) > 0)
    pick = touched[rng.choice(len(touched), size=min(60, len(touched)), replace=False)]
    fd, an = [], []
    for (r, c) in pick:
        Tp, Tm = T.copy(), T.copy()
        Tp[r, c] += h
        Tm[r, c] -= h
        fd.append((f(Tp, Ws) - f(Tm, Ws)) / (2 * h))
        an.append(dT[r, c])
    for i, W in enumerate(Ws):
        for idx in zip(*np.unravel_index(rng.choice(W.size, size=min(20, W.size), replace=False),
                                         W.shape)):
            Wp = [w_.copy() for w_ in Ws]
            Wm = [w_.copy() for w_ in Ws]
            Wp[i][idx] += h
            Wm[i][idx] -= h
            fd.append((f(T, Wp) - f(T, Wm)) / (2 * h))
            an.append(dWs[i][idx])
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd - an) <= 1e-6 * np.linalg.norm(an)
    # an untouched entry has zero gradient
    assert np.count_nonzero(dT) < dT.size
