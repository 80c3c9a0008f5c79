"""Pins of the oracle's training-regime functions (CPU only): the M-sample
target and loss of Eq. 3 / Eq. 14, the quarter schedule of Section 4 and the
first-intersection tracer of Eq. 2.  Each is checked against something other
than itself: the one-sample loss (already pinned), a hand-computed example,
central differences, duplicated samples, closed-form ray distances and a
brute-force FP64 ray march."""
import numpy as np
import pytest

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I


def _rand_loss_inputs(seed, N, M):
    g = np.random.default_rng(seed)
    Lp = g.uniform(0.05, 2.0, (N, 3))
    Ls = g.uniform(0.05, 2.0, (N, M, 3))
    E = g.uniform(0, 1, (N, 3)) * (g.random((N, 1)) < 0.3)
    w = g.uniform(0, 1, (N, M, 3))
    return Lp, Ls, E, w


@pytest.mark.parametrize("rhs_grad", [True, False])
def test_multi_loss_with_one_sample_is_the_one_sample_loss(rhs_grad):
    Lp, Ls, E, w = _rand_loss_inputs(1, 50, 1)
    a = O.residual_loss_multi(Lp, Ls, E, w, 1e-2, rhs_grad, 3.0)
    b = O.residual_loss(Lp, Ls[:, 0], E, w[:, 0], 1e-2, rhs_grad, 3.0)
    assert a[0] == pytest.approx(b[0], rel=1e-14)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-14)
    np.testing.assert_allclose(a[2][:, 0], b[2], rtol=1e-14, atol=0)


def test_multi_loss_duplicated_samples():
    """M copies of one sample give the one-sample target and loss; each copy
    receives 1/M of the one-sample gradient."""
    Lp, Ls, E, w = _rand_loss_inputs(2, 40, 1)
    M = 5
    a = O.residual_loss_multi(Lp, np.repeat(Ls, M, 1), E, np.repeat(w, M, 1), 1e-2, True)
    b = O.residual_loss(Lp, Ls[:, 0], E, w[:, 0], 1e-2, True)
    assert a[0] == pytest.approx(b[0], rel=1e-13)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-13)
    for m in range(M):
        np.testing.assert_allclose(a[2][:, m] * M, b[2], rtol=1e-13)


def test_multi_loss_hand_example():
    """N = 1, M = 2, the same value in all channels: L_p = 1, E = 0.5,
    w = (0.5, 1), L_s = (1, 2): T = 0.5 + (0.5 + 2) / 2 = 1.75, normaliser
    1 + 1.75 + 0.01 = 2.76, r = -0.75 / 2.76, loss = r^2."""
    Lp = np.ones((1, 3))
    E = np.full((1, 3), 0.5)
    w = np.array([[[0.5] * 3, [1.0] * 3]])
    Ls = np.array([[[1.0] * 3, [2.0] * 3]])
    loss, dLp, dLs = O.residual_loss_multi(Lp, Ls, E, w, 1e-2, True)
    r = -0.75 / 2.76
    assert loss == pytest.approx(r * r, rel=1e-15)
    np.testing.assert_allclose(dLp, np.full((1, 3), 2 * r / (3 * 2.76)), rtol=1e-14)
    np.testing.assert_allclose(dLs[0, 0], -dLp[0] * 0.5 / 2, rtol=1e-14)
    np.testing.assert_allclose(dLs[0, 1], -dLp[0] * 1.0 / 2, rtol=1e-14)


def test_multi_loss_gradient_by_central_differences():
    """The gradients equal central differences of the loss with its
    normaliser frozen (the stop-gradient of Eq. 14)."""
    N, M, eps = 6, 4, 1e-2
    Lp, Ls, E, w = _rand_loss_inputs(3, N, M)
    T0 = O.rhs_target(E, w, Ls)
    den0 = Lp + T0 + eps

    def frozen(Lp_, Ls_):
        r = (Lp_ - O.rhs_target(E, w, Ls_)) / den0
        return float(np.sum(r * r) / Lp_.size)
    _, dLp, dLs = O.residual_loss_multi(Lp, Ls, E, w, eps, True)
    h = 1e-6
    g = np.random.default_rng(4)
    for _ in range(10):
        i, c = int(g.integers(N)), int(g.integers(3))
        P, Q = Lp.copy(), Lp.copy()
        P[i, c] += h
        Q[i, c] -= h
        assert dLp[i, c] == pytest.approx((frozen(P, Ls) - frozen(Q, Ls)) / (2 * h), rel=1e-6)
        m = int(g.integers(M))
        P, Q = Ls.copy(), Ls.copy()
        P[i, m, c] += h
        Q[i, m, c] -= h
        assert dLs[i, m, c] == pytest.approx((frozen(Lp, P) - frozen(Lp, Q)) / (2 * h), rel=1e-6)


def test_quarter_schedule():
    total, n0, m0 = 100, 65536, 32
    got = [O.quarter_schedule(s, total, n0, m0) for s in range(total)]
    assert got[0] == got[24] == (65536, 32)
    assert got[25] == got[49] == (32768, 64)
    assert got[50] == got[74] == (16384, 128)
    assert got[75] == got[99] == (8192, 256)
    assert all(n * m == n0 * m0 for n, m in got)      # RHS samples per step stay fixed
    # ten steps: quarters are steps 0-2, 3-4, 5-7, 8-9 (q = floor(4 s / 10))
    assert [O.quarter_schedule(s, 10, 8, 1) for s in (2, 3, 4, 5, 7, 8, 9)] == \
        [(8, 1), (4, 2), (4, 2), (2, 4), (2, 4), (1, 8), (1, 8)]


# ------------------------------------------------------------------ tracer

NOPL = np.zeros((0, 13), np.float32)
NOSP = np.zeros((0, 4), np.float32)


def _plane(p, n, h):
    n = np.asarray(n, float) / np.linalg.norm(n)
    a = np.array([1.0, 0, 0]) if abs(n[0]) < 0.9 else np.array([0, 1.0, 0])
    t1 = np.cross(n, a)
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    return np.concatenate([p, n, t1, t2, [h]]).astype(np.float32)


def test_trace_box_walls():
    """From the box centre along the six axis directions the walls lie at
    t = 1/2 with ids P + S + 2a + (wall == 1)."""
    o = np.full((6, 3), 0.5, np.float32)
    d = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]], np.float32)
    t, prim, hit = O.trace_rays_f32(NOPL, NOSP, o, d, 1e-4)
    np.testing.assert_array_equal(t, np.full(6, 0.5, np.float32))
    np.testing.assert_array_equal(prim, np.arange(6))
    np.testing.assert_array_equal(hit, o + 0.5 * d)


def test_trace_sphere_and_patch_closed_forms():
    sp = np.array([[0.5, 0.5, 0.8, 0.1]], np.float32)
    pl = np.stack([_plane([0.5, 0.2, 0.5], [0, 1, 0], 0.1)])
    o = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5], [0.5, 0.5, 0.8], [0.5, 0.5, 0.5],
                  [0.65, 0.5, 0.5]], np.float32)
    d = np.array([[0, 0, 1], [0, -1, 0], [0, 0, 1], [0, 0, -1], [0, -1, 0]], np.float32)
    t, prim, _ = O.trace_rays_f32(pl, sp, o, d, 1e-4)
    # towards the sphere: t = 0.3 - 0.1; towards the patch: t = 0.3; from the
    # sphere's centre: its radius; away from both: the z = 0 wall; beside
    # the patch (|a| = 0.15 > 0.1): the y = 0 wall
    np.testing.assert_allclose(t, [0.2, 0.3, 0.1, 0.5, 0.5], rtol=1e-6)
    np.testing.assert_array_equal(prim, [1, 0, 1, 2 + 4, 2 + 2])


def _march(planes, spheres, o, d, t_min, step=1e-3, tmax=2.0):
    """Brute-force first crossing in FP64: sample the implicit functions of
    every primitive along the ray, take the first sign change (planes only
    where the crossing lies on the patch), refine it by bisection.  Returns
    (t, prim, margin): margin = distance of the decision from a tie or a
    patch edge, for excluding near-degenerate rays."""
    o = o.astype(np.float64)
    d = d.astype(np.float64)

    def pos(t):
        return o + np.multiply.outer(np.asarray(t, dtype=np.float64), d)
    funcs = []
    for k, pl in enumerate(planes.astype(np.float64)):
        funcs.append((k, lambda t, pl=pl: (pos(t) - pl[0:3]) @ pl[3:6], pl))
    P = len(planes)
    for s, sp in enumerate(spheres.astype(np.float64)):
        funcs.append((P + s, lambda t, sp=sp: np.sum((pos(t) - sp[0:3]) ** 2, -1) - sp[3] ** 2, None))
    S = len(spheres)
    for a in range(3):
        for wi, wall in enumerate((0.0, 1.0)):
            funcs.append((P + S + 2 * a + wi, lambda t, a=a, wall=wall: pos(t)[..., a] - wall, None))
    ts = np.arange(t_min, tmax, step)
    cands = []
    margin = np.inf
    for pid, fn, pl in funcs:
        v = fn(ts)
        sc = np.nonzero(np.sign(v[:-1]) * np.sign(v[1:]) < 0)[0]
        for i in sc:
            lo, hi = ts[i], ts[i + 1]
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                if np.sign(fn(mid)) == np.sign(fn(lo)):
                    lo = mid
                else:
                    hi = mid
            tc = 0.5 * (lo + hi)
            if pl is not None:
                rel = o + tc * d - pl[0:3]
                ea = max(abs(rel @ pl[6:9]), abs(rel @ pl[9:12])) - pl[12]
                margin = min(margin, abs(ea))
                if ea > 0:
                    continue
            cands.append((tc, pid))
            break
    cands.sort()
    if len(cands) > 1:
        margin = min(margin, cands[1][0] - cands[0][0])
    return cands[0][0], cands[0][1], margin


def test_trace_matches_brute_force_march():
    """Random rays from surface points of a patch scene: the binary32 tracer
    against the FP64 march (t to 1e-5, the same primitive), skipping rays
    whose decision lies within 1e-4 of a tie or a patch edge, or that graze
    a sphere (chord below the march step)."""
    g = I.rng(77)
    prims = I.make_primitives(g, 6, 6, patch=True)
    planes, spheres = I.scene_arrays(prims)
    o = g.uniform(0.05, 0.95, (150, 3)).astype(np.float32)
    d = I.unit_vectors(g, 150).astype(np.float32)
    t, prim, hit = O.trace_rays_f32(planes, spheres, o, d, 1e-4)
    checked = 0
    for i in range(len(o)):
        oc = o[i] - spheres[:, :3]
        b = oc @ d[i]
        disc = b * b - (np.sum(oc * oc, 1) - spheres[:, 3] ** 2)
        if np.any((disc > 0) & (disc < 1e-5)):
            continue
        tm, pm, margin = _march(planes, spheres, o[i], d[i], 1e-4)
        if margin < 1e-4:
            continue
        checked += 1
        assert prim[i] == pm, (i, prim[i], pm)
        assert abs(float(t[i]) - tm) <= 1e-5 * max(1.0, tm), (i, t[i], tm)
        np.testing.assert_allclose(hit[i], o[i] + t[i] * d[i], rtol=0, atol=1e-6)
    assert checked >= 120


def test_host_quarter_schedule_matches_oracle():
    """The library's host-side schedule against the oracle's."""
    from paper_2606_08469_gb300.train import quarter_schedule
    for total in (1, 3, 4, 10, 100, 20000):
        for s in sorted({0, 1, total // 4, total // 2, total - 1, max(0, total - 2)}):
            assert quarter_schedule(s, total, 65536, 32) == O.quarter_schedule(s, total, 65536, 32)
    with pytest.raises(ValueError):
        quarter_schedule(0, 0, 1, 1)
