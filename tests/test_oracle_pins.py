"""Pins of the FP64 oracle against things other than itself: published values,
closed forms, brute force, invariants and finite differences.  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import octaoctree_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------- RNG

def test_splitmix64_published_values():
    want = [int(r[0]) for r in _read_golden("splitmix64_seed1234567.txt")]
    s = 1234567
    got = []
    for _ in range(5):
        s, z = O.splitmix64_next(s)
        got.append(z)
    assert got == want


def test_splitmix64_unit_range():
    assert O.splitmix64_unit(0) == 0.0
    assert O.splitmix64_unit((1 << 64) - 1) == 1.0 - 2.0 ** -53


# ---------------------------------------------------------- paper arithmetic

def test_paper_storage_statistics():
    """Section 4.3: per-level node counts x (2^(9-l)+1)^2 vertices sum to the
    printed 79,375,000 entries; x 4 features x 4 B = 1211 MiB; Table 2's
    entry counts convert to its printed MB."""
    rows = _read_golden("table2_octaoctree_stats.txt")
    nodes = [r for r in rows if r[0] == "nodes"]
    counts = [int(r[4]) for r in nodes]
    sides = [int(r[3]) for r in nodes]
    for r in nodes:
        l = int(r[1])
        assert int(r[2]) == 2 ** (l + 1)      # spatial resolution 2^2 .. 2^9
        assert int(r[3]) == 2 ** (9 - l) + 1  # vertex resolution 2^8+1 .. 2^1+1
    total = [r for r in rows if r[0] == "total"][0]
    assert O.table_entries(counts, sides) == int(total[2])
    assert round(int(total[2]) * 4 * 4 / 2 ** 20) == int(total[3])
    for r in rows:
        if r[0] == "table2":
            mb = int(r[2]) * 4 * 4 / 2 ** 20
            assert abs(mb - float(r[3])) < 0.05 * (1 if float(r[3]) < 100 else 20)


# ------------------------------------------------------------------ octree

def _check_tree_structure(t):
    K = t.num_levels
    assert t.level_node_start[0] == 0 and t.level_node_start[K] == t.num_nodes
    for l in range(K):
        lo, hi = t.level_node_start[l], t.level_node_start[l + 1]
        assert np.all(t.node_level[lo:hi] == l)
    for n in range(t.num_nodes):
        fc = t.first_child[n]
        if fc >= 0:
            for b in range(8):
                c = t.node_coord[fc + b]
                bits = np.array([b & 1, (b >> 1) & 1, (b >> 2) & 1])
                assert np.array_equal(c, 2 * t.node_coord[n] + bits)
                assert t.node_level[fc + b] == t.node_level[n] + 1
    # map offsets: consecutive blocks of R_l^2 texels, levels back to back
    expect = 0
    for n in range(t.num_nodes):
        assert t.map_offset[n] == expect
        expect += t.R[t.node_level[n]] ** 2
    assert expect == t.num_texels


def test_tree_from_flags_by_hand():
    # root splits, then the 3rd child (slot 2: bx=0, by=1, bz=0) splits
    t = O.tree_from_flags([1, 0, 0, 1, 0, 0, 0, 0, 0], 2, [4, 2, 2])
    assert t.num_nodes == 1 + 8 + 8
    assert list(t.level_node_start) == [0, 1, 9, 17]
    assert t.first_child[0] == 1 and t.first_child[3] == 9
    assert list(t.node_coord[3]) == [0, 1, 0]
    assert list(t.node_coord[9 + 5]) == [1, 2, 1]  # slot 5 = bx 1, by 0, bz 1 under (0,1,0)
    assert t.num_texels == 16 + 8 * 4 + 8 * 4
    _check_tree_structure(t)


@pytest.mark.parametrize("seed,depth", [(1000, 4), (1001, 6), (7, 8)])
def test_seeded_tree_structure(seed, depth):
    R = [8] * (depth + 1)
    _check_tree_structure(O.build_tree(seed, depth, 0.6, R))


def test_tree_level_statistics():
    """E[N_l] = 8 N_{l-1} p^(l-1): 1, 8, 38.4, 110.6, 191.1 for p = 0.6."""
    counts = np.zeros(5)
    n_trees = 300
    for s in range(n_trees):
        t = O.build_tree(10_000 + s, 4, 0.6, [2] * 5)
        counts += np.diff(t.level_node_start)
    mean = counts / n_trees
    expect = [1.0]
    for l in range(1, 5):
        expect.append(expect[-1] * 8 * 0.6 ** (l - 1))
    assert mean[0] == 1 and mean[1] == 8
    for l in range(2, 5):
        assert abs(mean[l] - expect[l]) < 0.08 * expect[l], (l, mean[l], expect[l])


# ----------------------------------------------------------------- locate

def test_locate_matches_bruteforce():
    g = np.random.default_rng(0)
    for seed, depth in [(3, 3), (1000, 4), (1001, 6)]:
        t = O.build_tree(seed, depth, 0.6, [4] * (depth + 1))
        x = g.random((3000, 3)).astype(np.float32)
        # boundary points: cell faces at every level, 0 and 1
        edges = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5], [0.25, 0.75, 1.0],
                          [0.125, 0.0, 0.999999]], dtype=np.float32)
        x = np.concatenate([x, edges])
        assert np.array_equal(O.locate(t, x), O.locate_bruteforce(t, x))


def test_locate_exhaustive_tiny_tree():
    t = O.tree_from_flags([1, 1, 0, 0, 0, 0, 0, 0, 1], 2, [2, 2, 2])
    ax = (np.arange(8) + 0.5) / 8
    x = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    loc = O.locate(t, x)
    assert np.array_equal(loc, O.locate_bruteforce(t, x))
    # the root is everywhere; child 0 (x,y,z < 1/2) and child 7 are split
    assert np.all(loc[:, 0] == 0)
    deep = loc[:, 2] >= 0
    lo = np.all(x < 0.5, axis=1)
    hi = np.all(x >= 0.5, axis=1)
    assert np.array_equal(deep, lo | hi)


# ----------------------------------------------------------------- encode

def test_octa_encode_closed_forms():
    s2, s3 = math.sqrt(2), math.sqrt(3)
    w = np.array([[0, 0, 1], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, 0, -1],
                  [1 / s2, 1 / s2, 0], [1 / s3, 1 / s3, -1 / s3], [-1 / s3, 1 / s3, -1 / s3],
                  [0.6, -0.0, -0.8]])
    want = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [1, 1],
                     [0.5, 0.5], [2 / 3, 2 / 3], [-2 / 3, 2 / 3],
                     [1 - 0.0, (1 - 0.6 / 1.4)]])
    np.testing.assert_allclose(O.octa_encode(w), want, atol=1e-15)
    np.testing.assert_allclose(O.octa_uv(w)[0], [0.5, 0.5], atol=0)


def test_octa_round_trips():
    g = np.random.default_rng(1)
    w = g.normal(size=(20000, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    np.testing.assert_allclose(O.octa_decode(O.octa_encode(w)), w, atol=1e-14)
    u = g.uniform(-1, 1, size=(20000, 2))
    np.testing.assert_allclose(O.octa_encode(O.octa_decode(u)), u, atol=1e-13)
    # encode is onto the square and injective on a dense direction grid
    uu = O.octa_encode(w)
    assert np.all(np.abs(uu) <= 1 + 1e-15)


def test_octa_seam_identities():
    """(+-1, y) and (+-1, -y) are the same direction, likewise (x, +-1) and
    (-x, +-1); the four corners are (0,0,-1)."""
    y = np.linspace(-1, 1, 41)
    for sx in (-1.0, 1.0):
        a = O.octa_decode(np.stack([np.full_like(y, sx), y], 1))
        b = O.octa_decode(np.stack([np.full_like(y, sx), -y], 1))
        np.testing.assert_allclose(a, b, atol=1e-15)
        a = O.octa_decode(np.stack([y, np.full_like(y, sx)], 1))
        b = O.octa_decode(np.stack([-y, np.full_like(y, sx)], 1))
        np.testing.assert_allclose(a, b, atol=1e-15)
    c = O.octa_decode(np.array([[1, 1], [1, -1], [-1, 1], [-1, -1.0]]))
    np.testing.assert_allclose(c, np.tile([0, 0, -1.0], (4, 1)), atol=1e-15)


def test_corner_base_f32_matches_fp64_floor():
    g = np.random.default_rng(2)
    w = g.normal(size=(50000, 3)).astype(np.float32)
    for R in (2, 8, 16, 64):
        i0, j0 = O.corner_base_f32(w, R)
        p = O.octa_uv(w.astype(np.float64)) * R - 0.5
        ok = (np.abs(p[:, 0] - np.round(p[:, 0])) > 1e-4) & (np.abs(p[:, 1] - np.round(p[:, 1])) > 1e-4)
        assert ok.mean() > 0.99
        assert np.array_equal(i0[ok], np.floor(p[ok, 0]).astype(np.int64))
        assert np.array_equal(j0[ok], np.floor(p[ok, 1]).astype(np.int64))
        assert i0.min() >= -1 and i0.max() <= R - 1 and j0.min() >= -1 and j0.max() <= R - 1
    # closed forms: +z lands on texel centre corner (R/2-1, R/2-1) with f = 1/2
    i0, j0 = O.corner_base_f32(np.array([[0, 0, 1]], np.float32), 16)
    assert (i0[0], j0[0]) == (7, 7)
    i0, j0 = O.corner_base_f32(np.array([[0, 0, -1]], np.float32), 16)
    assert (i0[0], j0[0]) == (15, 15)          # corner uv = (1,1): p = 15.5


# ------------------------------------------------------------- wrap / blend

def test_wrap_tiny_exhaustive():
    for R in (2, 3, 4, 8):
        ii, jj = np.meshgrid(np.arange(-1, R + 1), np.arange(-1, R + 1), indexing="ij")
        wi, wj = O.wrap(ii.ravel(), jj.ravel(), R)
        assert wi.min() >= 0 and wi.max() < R and wj.min() >= 0 and wj.max() < R
        inside = (ii.ravel() >= 0) & (ii.ravel() < R) & (jj.ravel() >= 0) & (jj.ravel() < R)
        assert np.array_equal(wi[inside], ii.ravel()[inside])
        assert np.array_equal(wj[inside], jj.ravel()[inside])
    R = 4
    # diagonal corner rule and the edge mirror
    assert tuple(int(v[0]) for v in O.wrap([-1], [-1], R)) == (R - 1, R - 1)
    assert tuple(int(v[0]) for v in O.wrap([R], [R], R)) == (0, 0)
    assert tuple(int(v[0]) for v in O.wrap([R], [1], R)) == (R - 1, R - 2)
    assert tuple(int(v[0]) for v in O.wrap([1], [-1], R)) == (R - 2, 0)


def _single_node_tree(R):
    return O.tree_from_flags([], 0, [R])


def test_bilinear_partition_of_unity_and_constant():
    g = np.random.default_rng(3)
    t = O.build_tree(1000, 4, 0.6, [16, 16, 8, 8, 8])
    x = g.random((4000, 3)).astype(np.float32)
    w = g.normal(size=(4000, 3)).astype(np.float32)
    T = np.full((t.num_texels, 4), 0.37)
    enc = O.encode_features(t, T, x, w)
    present = enc.node >= 0
    np.testing.assert_allclose(enc.weight.sum(-1)[present], 1.0, atol=1e-12)
    assert enc.weight.min() > -1e-6 and enc.weight.max() < 1 + 1e-6
    h = enc.h.reshape(len(x), t.num_levels, 4)
    np.testing.assert_allclose(h[present], 0.37, atol=1e-12)
    np.testing.assert_array_equal(h[~present], 0.0)
    assert np.all(enc.addr[~present] == -1)


def test_bilinear_linear_table_closed_form():
    """Table value = a*(i+1/2)/R + b*(j+1/2)/R + c  =>  h = a*uv_x + b*uv_y + c
    wherever the 4 corners are inside the grid (texel centres, i along u_x)."""
    R = 8
    t = _single_node_tree(R)
    ij = np.arange(R * R)
    i, j = ij % R, ij // R
    a, b, c = 0.7, -1.3, 0.25
    T = (a * (i + 0.5) / R + b * (j + 0.5) / R + c)[:, None]
    g = np.random.default_rng(4)
    w = g.normal(size=(20000, 3)).astype(np.float32)
    x = np.full((len(w), 3), 0.5, np.float32)
    enc = O.encode_features(t, T, x, w)
    uv = O.octa_uv(w.astype(np.float64))
    p = uv * R - 0.5
    interior = np.all((p >= 0) & (p <= R - 1), axis=1)
    assert interior.mean() > 0.6
    np.testing.assert_allclose(enc.h[interior, 0], a * uv[interior, 0] + b * uv[interior, 1] + c,
                               atol=1e-12)


def test_features_continuous_across_seams():
    """A random table gives h(omega) continuous on the sphere: across the
    equator (Eq. 5's fold) and across the lower-hemisphere edges of the map."""
    R = 8
    t = _single_node_tree(R)
    g = np.random.default_rng(5)
    T = g.normal(size=(R * R, 3))
    x = np.full((1, 3), 0.3, np.float32)
    d = 1e-5
    worst = 0.0
    for _ in range(400):
        phi = g.uniform(0, 2 * np.pi)
        base = np.array([np.cos(phi), np.sin(phi), 0.0])
        # equator crossing
        cases = [(base + [0, 0, d], base - [0, 0, d])]
        # crossing the x-z half-plane below the equator (map edge u_y = 0 folded)
        th = g.uniform(0.05, np.pi / 2 - 0.05)
        sx = g.choice([-1.0, 1.0])
        b2 = np.array([sx * np.cos(th), 0.0, -np.sin(th)])
        cases.append((b2 + [0, d, 0], b2 - [0, d, 0]))
        b3 = np.array([0.0, sx * np.cos(th), -np.sin(th)])
        cases.append((b3 + [d, 0, 0], b3 - [d, 0, 0]))
        for p_, m_ in cases:
            w = np.stack([p_, m_]).astype(np.float32)
            h = O.encode_features(t, T, np.repeat(x, 2, 0), w).h
            worst = max(worst, float(np.abs(h[0] - h[1]).max()))
    assert worst < 1e-3, worst


def test_features_jump_without_wrap_detected():
    """Control for the continuity pin: clamping instead of wrapping makes h
    jump across the lower edges, so the pin above can fail."""
    R = 8
    g = np.random.default_rng(6)
    T = g.normal(size=(R * R,))
    w = np.array([[0.6, 1e-5, -0.8], [0.6, -1e-5, -0.8]])
    uv = O.octa_uv(w)
    p = uv * R - 0.5
    i0 = np.floor(p).astype(int)
    f = p - i0

    def clamp_blend(k):
        val = 0.0
        for a in (0, 1):
            for b in (0, 1):
                ii = min(max(i0[k, 0] + a, 0), R - 1)
                jj = min(max(i0[k, 1] + b, 0), R - 1)
                wt = (f[k, 0] if a else 1 - f[k, 0]) * (f[k, 1] if b else 1 - f[k, 1])
                val += wt * T[jj * R + ii]
        return val
    assert abs(clamp_blend(0) - clamp_blend(1)) > 1e-3


# -------------------------------------------------------------------- MLP

def test_mlp_closed_forms():
    # zero features -> exp(0) = 1
    Ws = [np.ones((4, 6)), np.ones((3, 4))]
    rgb, _, _ = O.mlp_forward(Ws, np.zeros((5, 6)))
    np.testing.assert_array_equal(rgb, 1.0)
    # hand network: z1 = [h0 - h1, h1], relu, out = exp([2 a0, -a1, a0 + a1])
    W1 = np.array([[1.0, -1.0], [0.0, 1.0]])
    W2 = np.array([[2.0, 0.0], [0.0, -1.0], [1.0, 1.0]])
    h = np.array([[0.5, 0.2], [0.1, 0.4], [-0.3, -0.2]])
    rgb, zs, _ = O.mlp_forward([W1, W2], h)
    a = np.maximum(np.stack([h[:, 0] - h[:, 1], h[:, 1]], 1), 0)
    np.testing.assert_allclose(rgb, np.exp(np.stack([2 * a[:, 0], -a[:, 1], a[:, 0] + a[:, 1]], 1)),
                               rtol=1e-15)


# -------------------------------------------------------------------- loss

def test_residual_loss_closed_forms():
    Lp = np.array([[1.0, 2.0, 0.5]])
    Ls = np.array([[0.5, 1.0, 2.0]])
    E = np.array([[0.5, 0.0, 0.0]])
    w = np.array([[1.0, 2.0, 0.25]])
    eps = 0.01
    # T = [1.0, 2.0, 0.5] == Lp: zero loss and zero gradient
    loss, dLp, dLs = O.residual_loss(Lp, Ls, E, w, eps)
    assert loss == 0.0 and not dLp.any() and not dLs.any()
    Lp2 = np.array([[2.0, 2.0, 0.5]])
    loss, dLp, dLs = O.residual_loss(Lp2, Ls, E, w, eps, rhs_grad=True, scale=4.0)
    r0 = (2.0 - 1.0) / (3.0 + eps)
    assert abs(loss - r0 * r0 / 3) < 1e-15
    assert abs(dLp[0, 0] - 4.0 * 2 * r0 / (3 * (3.0 + eps))) < 1e-14
    assert abs(dLs[0, 0] + 4.0 * 2 * r0 * 1.0 / (3 * (3.0 + eps))) < 1e-14
    _, _, dLs0 = O.residual_loss(Lp2, Ls, E, w, eps, rhs_grad=False)
    assert not dLs0.any()


def test_residual_loss_gradient_fd():
    """Gradient of the frozen-normaliser surrogate by central differences."""
    g = np.random.default_rng(7)
    Lp, Ls, E, w = (g.uniform(0.1, 2, size=(5, 3)) for _ in range(4))
    eps = 0.01
    _, dLp, dLs = O.residual_loss(Lp, Ls, E, w, eps)
    D0 = Lp + E + w * Ls

    def sur(Lp_, Ls_):
        return np.sum(((Lp_ - (E + w * Ls_)) / (D0 + eps)) ** 2) / Lp.size
    h = 1e-6
    for idx in np.ndindex(Lp.shape):
        e = np.zeros_like(Lp)
        e[idx] = h
        assert abs((sur(Lp + e, Ls) - sur(Lp - e, Ls)) / (2 * h) - dLp[idx]) < 1e-8
        assert abs((sur(Lp, Ls + e) - sur(Lp, Ls - e)) / (2 * h) - dLs[idx]) < 1e-8


# ---------------------------------------------------------------- backward

@pytest.mark.parametrize("rhs_grad", [True, False])
def test_backward_matches_finite_differences(rhs_grad):
    """Analytic table and weight gradients of the Eq. 14 loss vs central
    differences of its frozen-normaliser surrogate on 64 pairs."""
    from paper_2606_08469_gb300 import inputs as I
    t = O.build_tree(1000, 3, 0.6, [4, 4, 2, 2])
    F = 2
    g = np.random.default_rng(8)
    T = g.normal(0, 0.5, size=(t.num_texels, F))
    Ws = [W.astype(np.float64) for W in I.make_mlp(9, [t.num_levels * F, 8, 8, 3])]
    pairs = I.training_pairs(11, 64, 2, 2)
    N = pairs.n
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    rgb, _ = O.query_forward(t, T, Ws, X, Om)
    eps = 0.01
    loss, dLp, dLs = O.residual_loss(rgb[:N], rgb[N:], pairs.E, pairs.w, eps, rhs_grad)
    dT, dWs, _ = O.query_backward(t, T, Ws, X, Om, np.concatenate([dLp, dLs]))
    T0 = pairs.E + pairs.w * rgb[N:]
    D0 = rgb[:N] + T0

    def L(T_, Ws_):
        return O.surrogate_loss(t, T_, Ws_, pairs.x, pairs.omega, pairs.x2, -pairs.omega2,
                                pairs.E, pairs.w, D0, T0, eps, rhs_grad)
    assert abs(L(T, Ws) - loss) < 1e-15
    touched = np.nonzero(np.abs(dT).sum(1) > 0)[0]
    assert len(touched) > 20
    sel = g.choice(touched, size=min(40, len(touched)), replace=False)
    h = 1e-6
    for r in sel:
        for f in range(F):
            Tp, Tm = T.copy(), T.copy()
            Tp[r, f] += h
            Tm[r, f] -= h
            fd = (L(Tp, Ws) - L(Tm, Ws)) / (2 * h)
            assert abs(fd - dT[r, f]) <= 1e-7 * max(1e-3, abs(dT[r, f])) + 1e-10, (r, f, fd, dT[r, f])
    for li, W in enumerate(Ws):
        for idx in list(np.ndindex(W.shape))[::3]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[li][idx] += h
            Wm[li][idx] -= h
            fd = (L(T, Wp) - L(T, Wm)) / (2 * h)
            an = dWs[li][idx]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)) + 1e-10, (li, idx, fd, an)


# -------------------------------------------------------------------- Adam

def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-9, 0.0])
    p, m, v = O.adam_update(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_constant_gradient_closed_form():
    """For a constant gradient g, m_hat = g and v_hat = g^2 at every step."""
    g = np.array([0.5, -0.25])
    p, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    for t in range(1, 6):
        p, m, v = O.adam_update(p, g, m, v, t, lr=0.1, beta1=0.8, beta2=0.95, eps=0.0)
    np.testing.assert_allclose(p, -5 * 0.1 * np.sign(g), rtol=1e-12)


def test_loss_scaler_trajectory():
    s = O.LossScaler(scale=2.0 ** 15, growth_interval=3)
    seq = [True, False, True, True, True, True, False, False, True]
    skips, scales = [], []
    for finite in seq:
        skips.append(s.update(finite))
        scales.append(s.scale)
    assert skips == [False, True, False, False, False, False, True, True, False]
    assert scales == [2 ** 15, 2 ** 14, 2 ** 14, 2 ** 14, 2 ** 15, 2 ** 15, 2 ** 14, 2 ** 13, 2 ** 13]


def test_train_step_descends():
    """One Adam step with a small rate lowers the Eq. 14 surrogate loss."""
    from paper_2606_08469_gb300 import inputs as I
    t = O.build_tree(1000, 3, 0.6, [4, 4, 2, 2])
    T = np.random.default_rng(12).normal(0, 0.3, size=(t.num_texels, 4))
    Ws = [W.astype(np.float64) for W in I.make_mlp(13, [t.num_levels * 4, 16, 16, 3])]
    pairs = I.training_pairs(14, 256, 4, 4)
    st = O.TrainState(T.copy(), [w.copy() for w in Ws], np.zeros_like(T), np.zeros_like(T),
                      [np.zeros_like(w) for w in Ws], [np.zeros_like(w) for w in Ws])
    loss0, gn, skipped = O.train_step(t, st, pairs, O.LossScaler(), lr_tables=1e-4, lr_mlp=1e-4)
    assert not skipped and gn > 0
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    rgb0, _ = O.query_forward(t, T, Ws, X, Om)
    N = pairs.n
    T0 = pairs.E + pairs.w * rgb0[N:]
    D0 = rgb0[:N] + T0
    after = O.surrogate_loss(t, st.tables, st.weights, pairs.x, pairs.omega, pairs.x2, -pairs.omega2,
                             pairs.E, pairs.w, D0, T0, 0.01, True)
    assert after < loss0
