"""The training regime of Section 4 on the GPU against the oracle: the
secondary hits of Eq. 2 (octa_trace_rays, bit-exact: every decision in
binary32 in the same order), Eq. 3's M-sample target with Eq. 14
(residual_loss_multi, FP32 against FP64) and the whole M-sample training
step's gradients."""
import numpy as np
import pytest
import torch

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_08469_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _scene(seed, patch):
    g = I.rng(seed)
    prims = I.make_primitives(g, 8, 8, patch=patch)
    return g, prims, I.scene_arrays(prims)


@pytest.mark.parametrize("patch", [False, True])
def test_trace_bit_exact(patch):
    """Rays from surface points along hemisphere directions (the training
    case) and from random interior points along uniform directions, M = 7
    rays per origin: t, primitive and hit point bit for bit; query
    directions are the negated rays."""
    from paper_2606_08469_gb300 import api as A
    g, prims, (planes, spheres) = _scene(300 + patch, patch)
    xs, nrm = I.sample_surface_points(g, prims, 3000)
    M = 7
    d1 = I.hemisphere_directions(g, np.repeat(nrm, M, axis=0))
    xr = g.uniform(0.01, 0.99, (2000, 3))
    d2 = I.unit_vectors(g, 2000 * M)
    o = np.concatenate([xs, xr]).astype(np.float32)
    d = np.concatenate([d1, d2]).astype(np.float32)
    pr = A.Prims(planes, spheres, device=DEV)
    hit, qd, prim, t = A.octa_trace_rays(pr, dev(o), dev(d), M, 1e-4, query_dir=True,
                                         want_prim=True, want_t=True)
    rt, rp, rh = O.trace_rays_f32(planes, spheres, np.repeat(o, M, axis=0), d, 1e-4)
    np.testing.assert_array_equal(prim.cpu().numpy(), rp)
    np.testing.assert_array_equal(t.cpu().numpy(), rt)
    np.testing.assert_array_equal(hit.cpu().numpy(), rh)
    np.testing.assert_array_equal(qd.cpu().numpy(), -d)
    assert np.all(rp >= 0)                      # the box walls stop every ray


def test_trace_walls_only_edges_and_errors():
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    pr = A.Prims(np.zeros((0, 13)), np.zeros((0, 4)), device=DEV)
    o = np.array([[0.5, 0.5, 0.5], [0.0, 0.3, 0.7], [1e-6, 0.5, 0.5]], np.float32)
    d = np.array([[0, 0, 1], [1, 0, 0], [-1, 0, 0]], np.float32)
    hit, _, prim, t = A.octa_trace_rays(pr, dev(o), dev(d), 1, 1e-4, want_prim=True, want_t=True)
    rt, rp, rh = O.trace_rays_f32(np.zeros((0, 13)), np.zeros((0, 4)), o, d, 1e-4)
    np.testing.assert_array_equal(prim.cpu().numpy(), rp)
    np.testing.assert_array_equal(t.cpu().numpy(), rt)
    np.testing.assert_array_equal(hit.cpu().numpy(), rh)
    # the third ray's x = 0 wall lies within t_min and nothing else is ahead:
    # a miss (prim -1, t = inf)
    assert list(rp) == [5, 1, -1] and np.isinf(rt[2])
    A.octa_trace_rays(pr, dev(o)[:0], dev(d)[:0], 1)   # empty batch
    with pytest.raises(L.OctaError):
        A.octa_trace_rays(pr, dev(o), dev(d), 0)
    big = A.Prims(np.zeros((65, 13)), np.zeros((0, 4)), device=DEV)
    with pytest.raises(L.OctaError):
        A.octa_trace_rays(big, dev(o), dev(d), 1)


def _loss_inputs(seed, N, M):
    g = np.random.default_rng(seed)
    Lp = g.uniform(0.05, 2.0, (N, 3)).astype(np.float32)
    Ls = g.uniform(0.05, 2.0, (N, M, 3)).astype(np.float32)
    E = (g.uniform(0, 1, (N, 3)) * (g.random((N, 1)) < 0.1)).astype(np.float32)
    w = g.uniform(0, 1, (N, M, 3)).astype(np.float32)
    return Lp, Ls, E, w


@pytest.mark.parametrize("M", [1, 3, 32, 37, 256])
@pytest.mark.parametrize("rhs_grad", [True, False])
def test_loss_multi_matches_oracle(M, rhs_grad):
    """FP32 against FP64: the loss to 1e-5 relative, the gradients to 1e-5
    normwise (the per-channel sums over M run in FP32 with two partial
    sums; 256 terms of products in [0, 2] stay well inside 1e-5)."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    N = 2049
    Lp, Ls, E, w = _loss_inputs(M + 7 * rhs_grad, N, M)
    dLp = torch.empty((N, 3), device=DEV)
    dLs = torch.full((N, M, 3), 7.0, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    ws = A.workspace(L.OCTA_OP_LOSS, N, device=DEV)
    A.residual_loss_multi(dev(Lp), dev(Ls), dev(E), dev(w), dLp, dLs, loss, ws, 1e-2, rhs_grad)
    ref, rLp, rLs = O.residual_loss_multi(Lp, Ls, E, w, 1e-2, rhs_grad)
    assert abs(loss.item() - ref) <= 1e-5 * ref
    gp = dLp.cpu().numpy()
    assert np.linalg.norm(gp - rLp) <= 1e-5 * np.linalg.norm(rLp)
    gs = dLs.cpu().numpy()
    if rhs_grad:
        assert np.linalg.norm(gs - rLs) <= 1e-5 * np.linalg.norm(rLs)
    else:
        assert np.all(gs == 0)


def test_loss_multi_with_one_sample_equals_residual_loss():
    """M = 1 evaluates residual_loss's formulas; there T = E + w L_s is one
    fused multiply-add, here the product is rounded first, so values agree
    to binary32 rounding (gradients 1e-6 normwise, the loss 1e-7)."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    N = 5000
    Lp, Ls, E, w = _loss_inputs(11, N, 1)
    out = []
    for multi in (True, False):
        dLp = torch.empty((N, 3), device=DEV)
        dLs = torch.empty((N, 3), device=DEV)
        loss = torch.zeros(1, dtype=torch.float64, device=DEV)
        ws = A.workspace(L.OCTA_OP_LOSS, N, device=DEV)
        if multi:
            A.residual_loss_multi(dev(Lp), dev(Ls), dev(E), dev(w), dLp, dLs.view(N, 1, 3), loss,
                                  ws, 1e-2, True)
        else:
            A.residual_loss(dev(Lp), dev(Ls[:, 0]), dev(E), dev(w[:, 0]), dLp, dLs, loss, ws, 1e-2,
                            True)
        out.append((loss.item(), dLp.cpu().numpy(), dLs.cpu().numpy()))
    assert out[0][0] == pytest.approx(out[1][0], rel=1e-7)
    for k in (1, 2):
        assert np.linalg.norm(out[0][k] - out[1][k]) <= 1e-6 * np.linalg.norm(out[1][k])


@pytest.mark.parametrize("rhs_grad", [False, True])
def test_multi_sample_step_gradients_match_oracle(rhs_grad):
    """One M-sample training step of the FP32 train_f32 scene (300
    LHS samples, M = 8): the traced secondaries are the oracle's bit for bit,
    and the table / decoder gradients (before Adam) agree with the oracle's
    FP64 forward, M-sample loss and backward to 1e-5 normwise."""
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_f32"]
    step, (tree, tables, weights, smp) = WL.multi_sample_step_for(
        cfg, 300, 8, device=DEV, precision="f32", rhs_grad=rhs_grad, scale=1.0,
        growth_interval=0)
    step.trace()
    step.forward()
    step.loss_and_grad()
    step.backward()
    torch.cuda.synchronize()
    N, M = smp.n, smp.M
    _, _, hit = O.trace_rays_f32(smp.planes, smp.spheres, np.repeat(smp.x, M, axis=0),
                                 smp.omega_i.reshape(-1, 3), 1e-4)
    np.testing.assert_array_equal(step.X[N:].cpu().numpy(), hit)
    ot = O.build_tree(cfg.seed("tree"), cfg.max_depth, cfg.p_base, cfg.R)
    X = np.concatenate([smp.x, hit])
    Om = np.concatenate([smp.omega, -smp.omega_i.reshape(-1, 3)])
    rgb, _ = O.query_forward(ot, tables, weights, X, Om)
    loss, dLp, dLs = O.residual_loss_multi(rgb[:N], rgb[N:].reshape(N, M, 3), smp.E, smp.w,
                                           1e-2, rhs_grad)
    assert abs(step.loss.item() - loss) <= 1e-5 * loss
    d_rgb = np.concatenate([dLp, dLs.reshape(-1, 3)])
    rT, rWs, _ = O.query_backward(ot, tables, weights, X, Om, d_rgb)
    gT = step.state.grad_t.cpu().numpy()
    assert np.linalg.norm(gT - rT) <= 1e-5 * np.linalg.norm(rT)
    gw = step.state.grad_w.cpu().numpy()
    for (off, o, i), rW in zip(step.scene.weight_slices(), rWs):
        assert np.linalg.norm(gw[off:off + o * i].reshape(o, i) - rW) <= 1e-5 * np.linalg.norm(rW)
    step.optimizer()
    step.step()
    torch.cuda.synchronize()
    assert np.isfinite(step.loss.item())


def test_full_size_quarter0_samples():
    """The bench's first quarter at full size (train_bf16's scene and BF16
    decoder, 65,536 LHS samples x M = 32): 2,000 sampled secondary hits
    bit-exact against the oracle's tracer, the loss equal to the oracle's
    M-sample loss evaluated on the GPU's radiances (FP64, 1e-6), and 300
    sampled radiances within the BF16 path's 1e-2 normwise bound."""
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_bf16"]
    step, (tree, tables, weights, smp) = WL.multi_sample_step_for(cfg, 65536, 32, device=DEV)
    step.trace()
    step.forward()
    step.loss_and_grad()
    torch.cuda.synchronize()
    N, M = smp.n, smp.M
    g = np.random.default_rng(3)
    rays = g.choice(N * M, 2000, replace=False)
    o = smp.x[rays // M]
    d = smp.omega_i.reshape(-1, 3)[rays]
    _, _, hit = O.trace_rays_f32(smp.planes, smp.spheres, o, d, 1e-4)
    np.testing.assert_array_equal(step.X[N:].cpu().numpy()[rays], hit)
    rgb = step.rgb.cpu().numpy().astype(np.float64)
    loss, _, _ = O.residual_loss_multi(rgb[:N], rgb[N:].reshape(N, M, 3), smp.E, smp.w, 1e-2, False)
    assert abs(step.loss.item() - loss) <= 1e-6 * loss
    rows = g.choice(N + N * M, 300, replace=False)
    X = step.X.cpu().numpy()[rows]
    Om = step.Om.cpu().numpy()[rows]
    ot = O.build_tree(cfg.seed("tree"), cfg.max_depth, cfg.p_base, cfg.R)
    ref, _ = O.query_forward(ot, tables, weights, X, Om)
    assert np.linalg.norm(rgb[rows] - ref) <= 1e-2 * np.linalg.norm(ref)
