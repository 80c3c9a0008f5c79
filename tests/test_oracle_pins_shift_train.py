"""Pins of the oracle's training of the disparity predictor through the
shifted lookup (CPU only): a query's dL/dd (disparity_gradient) against
central differences in d, and a whole training step's g_psi gradients
(shifted_train_gradients) against central differences of the step's loss in
g_psi's weights and hash entries (the normaliser of Eq. 14 frozen, as its
stop-gradient prescribes).

Every lookup decides its cells' triangles in binary32, so a step in d or in
psi must move d by far more than a binary32 ulp; the steps here move d by
1e-3 relative in the per-query test (queries whose binary32 decisions or
ReLU masks change across the step left out) and about 1e-4 in the step's
(where the difference quotient has converged to within 1e-3 of its limit),
and the tolerances (3e-3 per query normwise, 1e-2 for the step) reflect
that resolution.  A dropped factor, a wrong sign or a transposed Jacobian is off
by O(1)."""
import numpy as np
import pytest

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I

F32 = np.float32


def _queries(seed, n):
    g = I.rng(seed)
    x = g.random((n, 3)).astype(F32)
    w = I.unit_vectors(g, n).astype(F32)
    nrm = I.unit_vectors(g, n).astype(F32)
    return x, w, nrm, g


def _masks(weights, h):
    a = np.asarray(h, np.float64)
    out = []
    for W in weights[:-1]:
        z = a @ np.asarray(W, np.float64).T
        out.append(z > 0)
        a = np.maximum(z, 0.0)
    return np.concatenate(out, axis=1)


@pytest.mark.parametrize("with_attrs", [False, True])
def test_disparity_gradient_by_central_differences(with_attrs):
    ot = O.build_tree(91, 3, 0.8, [17, 9, 9, 5])
    tables = I.make_tables(92, ot.num_texels, 4, 0.5)
    n = 400
    x, w, nrm, g = _queries(93, n)
    d = g.uniform(0.5, 4.0, n).astype(F32)
    n_attrs = 5 if with_attrs else 0
    attrs = g.normal(size=(n, n_attrs)) if with_attrs else None
    weights = [W * F32(2.0) for W in I.make_mlp(94, [16 + n_attrs, 16, 16, 3])]
    c = g.normal(size=(n, 3))
    an = O.disparity_gradient(ot, tables, weights, x, w, nrm, d, c, attrs=attrs)

    def run(dd):
        rgb, enc = O.query_forward(ot, tables, weights, x, w, form="shifted", normal=nrm,
                                   disparity=dd, attrs=attrs)
        return np.sum(c * rgb, axis=1), enc, _masks(weights, O.decoder_input(enc.h, attrs))
    dp = (d * F32(1.001)).astype(F32)
    dm = (d * F32(0.999)).astype(F32)
    fp, ep, mp = run(dp)
    fm, em, mm = run(dm)
    _, e0, m0 = run(d)
    same = np.all((ep.addr == e0.addr) & (em.addr == e0.addr), axis=(1, 2, 3))
    same &= np.all((mp == m0) & (mm == m0), axis=1)
    assert same.sum() > n // 3
    fd = (fp - fm) / (dp.astype(np.float64) - dm.astype(np.float64))
    assert np.linalg.norm(fd[same]) > 0
    assert np.linalg.norm(an[same] - fd[same]) <= 3e-3 * np.linalg.norm(fd[same])


def _step_case(rhs_grad):
    ot = O.build_tree(95, 3, 0.8, [17, 9, 9, 5])
    tables = I.make_tables(96, ot.num_texels, 4, 0.5)
    weights = [W * F32(1.5) for W in I.make_mlp(97, [16, 16, 16, 3])]
    levels = 4
    res = O.hash_resolutions(levels, 4, 14)
    ptab, pw = I.predictor_params(98, levels, 10, table_scale=0.5)
    pw = [W * F32(2.0) for W in pw]
    pairs, n1, n2 = I.training_pairs_with_normals(99, 250)
    return ot, tables, weights, (ptab, res, pw), pairs, n1, n2


@pytest.mark.parametrize("rhs_grad", [True, False])
def test_shifted_step_gradients_by_central_differences(rhs_grad):
    ot, tables, weights, pred, pairs, n1, n2 = _step_case(rhs_grad)
    ptab, res, pw = pred
    eps = 1e-2
    loss, dT, dWs, dtab, dWp, dd, d = O.shifted_train_gradients(
        ot, tables, weights, pred, pairs, n1, n2, eps=eps, rhs_grad=rhs_grad)
    n = pairs.n
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    Nr = np.concatenate([n1, n2])
    E = pairs.E.astype(np.float64)
    wt = pairs.w.astype(np.float64)

    def radiance(tab, Ws):
        dq = O.disparity(tab, res, Ws, X, Om, Nr).astype(F32)
        rgb, _ = O.query_forward(ot, tables, weights, X, Om, form="shifted", normal=Nr,
                                 disparity=dq)
        return rgb
    rgb0 = radiance(ptab, pw)
    T0 = E + wt * rgb0[n:]
    D0 = rgb0[:n] + T0

    def surrogate(tab, Ws):
        rgb = radiance(tab, Ws)
        T = E + wt * rgb[n:] if rhs_grad else T0
        r = (rgb[:n] - T) / (D0 + eps)
        return float(np.sum(r * r) / r.size)
    assert surrogate(ptab, pw) == pytest.approx(loss, rel=1e-12)
    rng = np.random.default_rng(100)

    def fd_weight(i, a, b, h=1e-4):
        P = [W.astype(np.float64) for W in pw]
        Q = [W.astype(np.float64) for W in pw]
        P[i][a, b] += h
        Q[i][a, b] -= h
        return (surrogate(ptab, P) - surrogate(ptab, Q)) / (2 * h)

    def fd_entry(l, t, f, h=1e-4):
        P = ptab.astype(np.float64).copy()
        Q = ptab.astype(np.float64).copy()
        P[l, t, f] += h
        Q[l, t, f] -= h
        return (surrogate(P, pw) - surrogate(Q, pw)) / (2 * h)
    # compared normwise per group (a component near zero is as exact as the
    # group's scale allows): the last layer, where every query's d moves by
    # a factor exp(+-h a_k); first-layer weights on the hash features and
    # omega_r's components; the busiest hash entries
    groups = []
    ks = rng.choice(64, 6, replace=False)
    groups.append(([dWp[2][0, k] for k in ks], [fd_weight(2, 0, k) for k in ks]))
    cols = [0, 3, 8, 9, 10]
    rows = [int(np.argmax(np.abs(dWp[0][:, c]))) for c in cols]
    groups.append(([dWp[0][r, c] for r, c in zip(rows, cols)],
                   [fd_weight(0, r, c) for r, c in zip(rows, cols)]))
    ents = [np.unravel_index(e, dtab.shape) for e in np.argsort(np.abs(dtab).ravel())[::-1][:4]]
    groups.append(([dtab[e] for e in ents], [fd_entry(*e) for e in ents]))
    for an, fd in groups:
        an, fd = np.array(an), np.array(fd)
        assert np.linalg.norm(fd) > 0
        assert np.linalg.norm(an - fd) <= 1e-2 * np.linalg.norm(fd), (an, fd)


def test_shifted_step_reduces_to_its_parts():
    """The step's decoder and table gradients are query_backward's on the
    Eq. 14 gradient at the predicted (binary32) disparity, and its g_psi
    gradients are disparity_backward's on that disparity gradient."""
    ot, tables, weights, pred, pairs, n1, n2 = _step_case(True)
    ptab, res, pw = pred
    loss, dT, dWs, dtab, dWp, dd, d = O.shifted_train_gradients(ot, tables, weights, pred, pairs,
                                                                n1, n2, scale=4.0)
    n = pairs.n
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    Nr = np.concatenate([n1, n2])
    np.testing.assert_allclose(d, O.disparity(ptab, res, pw, X, Om, Nr), rtol=0)
    rgb, _ = O.query_forward(ot, tables, weights, X, Om, form="shifted", normal=Nr,
                             disparity=d.astype(F32))
    l2, dLp, dLs = O.residual_loss(rgb[:n], rgb[n:], pairs.E, pairs.w, scale=4.0)
    assert l2 == loss
    d_rgb = np.concatenate([dLp, dLs])
    rT, rWs, _ = O.query_backward(ot, tables, weights, X, Om, d_rgb, form="shifted", normal=Nr,
                                  disparity=d.astype(F32))
    np.testing.assert_allclose(dT, rT, rtol=1e-12, atol=1e-15)
    rdd = O.disparity_gradient(ot, tables, weights, X, Om, Nr, d, d_rgb)
    np.testing.assert_allclose(dd, rdd, rtol=1e-12, atol=1e-15)
    rtab, rWp = O.disparity_backward(ptab, res, pw, X, Om, Nr, dd)
    np.testing.assert_allclose(dtab, rtab, rtol=1e-12, atol=1e-15)
    for a, b in zip(dWp, rWp):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15)
