"""The full query form on the GPU (OCTA_FORM_TRILINEAR_VERTEX: Eq. 10
eight-cell renormalised trilinear blend with Eq. 6 barycentric interpolation
on vertex maps) against the FP64 oracle: the 24 vertex entries per level
bit-exact, features within the binary32 bound of a 24-term blend; the FP32
decoder's forward, backward and fused training pass in the same form."""
import numpy as np
import pytest
import torch

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"
U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_08469_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _scene(tree, tables, tdt=torch.float32):
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    F = tables.shape[1]
    weights = [dev(W) for W in I.make_mlp(1, [tree.num_levels * F, 16, 3])]
    return A.Scene(tree, dev(tables).to(tdt).contiguous(), weights, device=DEV,
                   query_form=L.OCTA_FORM_TRILINEAR_VERTEX)


def _check(tree, ot, tables, x, w, tdt=torch.float32):
    from paper_2606_08469_gb300 import api as A
    sc = _scene(tree, tables, tdt)
    tq = tables.astype(np.float16).astype(np.float64) if tdt == torch.float16 else tables
    feat, _, addr = A.octa_encode(sc, dev(x), dev(w), want_addr=True)
    ref = O.encode_features_full(ot, tq, x, w)
    K = tree.num_levels
    np.testing.assert_array_equal(addr.cpu().numpy(), ref.addr.reshape(len(x), K, 24))
    bound = 64 * U32 * np.abs(tq).max()
    np.testing.assert_allclose(feat.cpu().numpy(), ref.h, rtol=1e-6, atol=bound)
    fb, _, _ = A.octa_encode(sc, dev(x), dev(w), feat_dtype=torch.bfloat16)
    np.testing.assert_allclose(fb.float().cpu().numpy(), ref.h, rtol=2 ** -8, atol=bound)
    return ref


@pytest.mark.parametrize("seed,depth,V,F,tdt", [
    (1200, 4, [9, 9, 5, 5, 3], 4, torch.float32),
    (1201, 6, [17, 17, 9, 9, 5, 5, 3], 8, torch.float16),
    (1202, 2, [3, 5, 9], 8, torch.float32),
])
def test_full_form_random_trees(seed, depth, V, F, tdt):
    from paper_2606_08469_gb300 import api as A
    tree = A.octree_build(seed, depth, 0.6, V)
    ot = O.build_tree(seed, depth, 0.6, V)
    tables = I.make_tables(seed + 1, tree.num_texels, F, 0.3)
    x, w = I.uniform_queries(seed + 2, 5000)
    _check(tree, ot, tables, x, w, tdt)


def test_full_form_edges_dense_tree_and_seams():
    """Dense depth-3 tree; positions on the cube's faces and corners and on
    cell boundaries, directions on the fold's edges and the octahedron's
    vertices."""
    from paper_2606_08469_gb300 import api as A
    V = [5, 5, 3, 3]
    tree = A.octree_build(7, 3, 1.0, V)
    ot = O.build_tree(7, 3, 1.0, V)
    tables = I.make_tables(8, tree.num_texels, 4, 0.5)
    g = np.random.default_rng(9)
    xs = [np.zeros(3), np.ones(3), np.full(3, 0.5), np.array([0.125, 0.375, 1.0]),
          np.array([0.0, 0.9375, 0.0625])]
    ws = [np.array(v, float) for v in ([0, 0, 1], [0, 0, -1], [1, 0, 0], [0, -1, 0], [1, 1, 0],
                                         [1, -1, -1e-7], [-0.3, 0.0, -0.7], [0.5, -0.5, 0.0])]
    x = np.array([a for a in xs for _ in ws] + list(g.random((600, 3))), np.float32)
    w = np.array([b for _ in xs for b in ws] + list(g.normal(size=(600, 3))), np.float32)
    _check(tree, ot, tables, x, w)


def test_full_form_sparse_tree_zero_levels():
    from paper_2606_08469_gb300 import api as A
    flags = [1, 1, 0, 0, 0, 0, 0, 0, 0]
    V = [3, 5, 3]
    tree = A.octree_from_flags(flags, 2, V)
    ot = O.tree_from_flags(flags, 2, V)
    tables = I.make_tables(3, tree.num_texels, 4, 0.5)
    x, w = I.uniform_queries(4, 3000)
    ref = _check(tree, ot, tables, x, w)
    assert np.any(ref.h[:, 8:12] == 0) and np.any(ref.h[:, 8:12] != 0)


def test_full_form_global_walk():
    """A 4,681-node tree: more than the staged-tree capacity."""
    from paper_2606_08469_gb300 import api as A
    V = [3, 3, 3, 3, 3]
    tree = A.octree_build(5, 4, 1.0, V)
    assert tree.num_nodes > 2048
    ot = O.build_tree(5, 4, 1.0, V)
    tables = I.make_tables(6, tree.num_texels, 4, 0.3)
    x, w = I.uniform_queries(7, 3000)
    _check(tree, ot, tables, x, w)


def test_full_form_argument_errors():
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    tree = A.octree_build(5, 2, 0.6, [4, 3, 3])       # 4 is not 2^k + 1
    sc = _scene(tree, I.make_tables(1, tree.num_texels, 4, 0.3))
    x, w = I.uniform_queries(1, 10)
    with pytest.raises(L.OctaError):
        A.octa_encode(sc, dev(x), dev(w))
    tree = A.octree_build(5, 2, 0.6, [5, 3, 3])
    sc = _scene(tree, I.make_tables(1, tree.num_texels, 4, 0.3))
    with pytest.raises(L.OctaError):
        A.octa_encode(sc, dev(x), dev(w), want_nodes=True)
    with pytest.raises(L.OctaError):
        A.octa_query_fwd(sc, dev(x), dev(w), want_nodes=True)
    weights = [dev(W).to(torch.bfloat16) for W in I.make_mlp(1, [12, 32, 32, 3])]
    sb = A.Scene(tree, sc.tables, weights, device=DEV, query_form=L.OCTA_FORM_TRILINEAR_VERTEX)
    A.octa_encode(sb, dev(x), dev(w))                     # the encoding and the forward take
    A.octa_query_fwd(sb, dev(x), dev(w))                  # either decoder
    cell = A.Scene(tree, sc.tables, [dev(W) for W in I.make_mlp(1, [12, 16, 3])], device=DEV)
    two = [sc, cell]                                      # forms mixed in one call
    with pytest.raises(L.OctaError):
        A.octa_query_fwd(two, dev(np.concatenate([x, x])), dev(np.concatenate([w, w])), [10, 10])


# ------------------------------------------- FP32 decoder passes (FP32 engine)

def _decoder_scene(seed, depth, V, F, hidden, tdt=torch.float32, wscale=1.5):
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    tree = A.octree_build(seed, depth, 0.6, V)
    ot = O.build_tree(seed, depth, 0.6, V)
    tables = I.make_tables(seed + 1, tree.num_texels, F, 0.3)
    if tdt == torch.float16:
        tables = tables.astype(np.float16).astype(np.float32)   # the values the GPU reads
    weights = [W * np.float32(wscale) for W in I.make_mlp(seed + 2, [(depth + 1) * F] + hidden + [3])]
    sc = A.Scene(tree, dev(tables).to(tdt).contiguous(), [dev(W) for W in weights], device=DEV,
                 query_form=L.OCTA_FORM_TRILINEAR_VERTEX)
    return sc, ot, tables, weights


def _rgb_tol(ot, tables, weights, x, w):
    """|rgb_gpu / rgb - 1| bound: the absolute error of z, at most c * u *
    z_abs with z_abs the decoder run on |W| and on the blend of |tables|
    (the 24 blend weights are non-negative, so that blend bounds the
    features' rounding as well); c = 16 as for the cell form, floor 1e-5."""
    habs = O.encode_features_full(ot, np.abs(tables), x, w).h
    _, zs, _ = O.mlp_forward([np.abs(W) for W in weights], habs)
    return np.maximum(1e-5, 16 * U32 * zs[-1])


def _normwise(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


FP32_SCENES = [
    (1300, 4, [9, 9, 5, 5, 3], 4, [32, 32], torch.float32),
    (1301, 5, [17, 17, 9, 9, 5, 3], 8, [64, 64], torch.float16),
    (1302, 6, [9, 9, 9, 5, 5, 3, 3], 8, [64, 64, 64], torch.float32),
]
WSCALE = {1300: 1.5, 1301: 1.5, 1302: 0.5}   # three hidden layers: keep z_abs moderate


@pytest.mark.parametrize("seed,depth,V,F,hidden,tdt", FP32_SCENES)
def test_full_form_query_fwd_matches_oracle(seed, depth, V, F, hidden, tdt):
    """octa_query_fwd on an FP32 decoder in the full form: radiance within
    the FP32 bound, the 24 entries of every level bit-exact, on a ragged
    batch (several 128-query tiles and a tail)."""
    from paper_2606_08469_gb300 import api as A
    sc, ot, tables, weights = _decoder_scene(seed, depth, V, F, hidden, tdt, WSCALE[seed])
    x, w = I.uniform_queries(seed + 3, 3001)
    rgb, _, addr = A.octa_query_fwd(sc, dev(x), dev(w), want_addr=True)
    ref, enc = O.query_forward(ot, tables, weights, x, w, form="full")
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr.reshape(len(x), depth + 1, 24))
    err = np.abs(rgb.cpu().numpy() - ref) / ref
    assert np.all(err <= _rgb_tol(ot, tables, weights, x, w)), err.max()


@pytest.mark.parametrize("seed,depth,V,F,hidden,tdt", FP32_SCENES[:2])
def test_full_form_query_bwd_matches_oracle(seed, depth, V, F, hidden, tdt):
    """octa_query_bwd in the full form: the 24 entries of a level each
    receive (renormalised cell weight x barycentric) x dh; table and weight
    gradients to 1e-5 normwise against the FP64 oracle."""
    from paper_2606_08469_gb300 import api as A
    sc, ot, tables, weights = _decoder_scene(seed, depth, V, F, hidden, tdt)
    x, w = I.uniform_queries(seed + 4, 4000)
    d_rgb = np.random.default_rng(seed).normal(size=(len(x), 3)).astype(np.float32)
    dT = torch.zeros((sc.tree.num_texels, F), device=DEV)
    dW = torch.zeros(sc.weights.shape, device=DEV)
    A.octa_query_bwd(sc, dev(x), dev(w), dev(d_rgb), [(dT, dW)])
    rT, rWs, _ = O.query_backward(ot, tables, weights, x, w, d_rgb, form="full")
    assert _normwise(dT.cpu().numpy(), rT) <= 1e-5
    gw = dW.cpu().numpy()
    for (off, o, i), rW in zip(sc.weight_slices(), rWs):
        assert _normwise(gw[off:off + o * i].reshape(o, i), rW) <= 1e-5


@pytest.mark.parametrize("rhs_grad", [True, False])
def test_full_form_fused_training_matches_oracle(rhs_grad):
    """octa_train_fused (FP32 engine, 64-pair tiles) in the full form: the
    Eq. 14 loss to 1e-5 and the gradients of both queries of every pair to
    1e-5 normwise, against the oracle's residual_loss and query_backward on
    the same pairs (1,001 pairs: a ragged tail tile)."""
    from paper_2606_08469_gb300 import api as A
    seed, depth, V, F, hidden, tdt = FP32_SCENES[1]
    sc, ot, tables, weights = _decoder_scene(seed, depth, V, F, hidden, tdt)
    pr = I.training_pairs(seed + 5, 1001)
    dT = torch.zeros((sc.tree.num_texels, F), device=DEV)
    dW = torch.zeros(sc.weights.shape, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    A.octa_train_fused(sc, dev(pr.x), dev(pr.omega), dev(pr.x2), dev(-pr.omega2), dev(pr.E),
                       dev(pr.w), [(dT, dW)], loss, rhs_grad=rhs_grad)
    N = len(pr.x)
    X = np.concatenate([pr.x, pr.x2])
    Om = np.concatenate([pr.omega, -pr.omega2])
    rgb, _ = O.query_forward(ot, tables, weights, X, Om, form="full")
    ref_loss, dLp, dLs = O.residual_loss(rgb[:N], rgb[N:], pr.E, pr.w, 1e-2, rhs_grad)
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    rT, rWs, _ = O.query_backward(ot, tables, weights, X, Om, np.concatenate([dLp, dLs]),
                                  form="full")
    assert _normwise(dT.cpu().numpy(), rT) <= 1e-5
    gw = dW.cpu().numpy()
    for (off, o, i), rW in zip(sc.weight_slices(), rWs):
        assert _normwise(gw[off:off + o * i].reshape(o, i), rW) <= 1e-5


def test_full_form_train_step_fused_matches_unfused():
    """The training step of the headline workload's shapes (FP32, 2,049
    pairs) in the full form: the fused pass against octa_query_fwd +
    residual_loss + octa_query_bwd, then one Adam step each."""
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_f32"]
    a, _ = WL.train_step_for(cfg, n_pairs=2049, precision="f32", query_form="full")
    b, _ = WL.train_step_for(cfg, n_pairs=2049, precision="f32", query_form="full", fused=True)
    a.forward()
    a.loss_and_grad()
    a.backward()
    b.fused_pass()
    torch.cuda.synchronize()
    torch.testing.assert_close(b.loss, a.loss, rtol=1e-6, atol=0)
    for sa, sb in zip(a.states, b.states):
        for ga, gb in ((sa.grad_t, sb.grad_t), (sa.grad_w, sb.grad_w)):
            assert (torch.linalg.norm(gb - ga) / torch.linalg.norm(ga)).item() <= 1e-5
    a.step()
    b.step()
    torch.cuda.synchronize()
    assert np.isfinite(a.loss.item()) and np.isfinite(b.loss.item())


@pytest.mark.parametrize("tdt", [torch.float16, torch.float32])
def test_full_form_tensor_core_forward(tdt):
    """The tcgen05 forward (BF16 decoder 48-64-64-3) in the full form on a
    ragged batch: the 24 entries of every level bit-exact, radiance within
    the BF16 path's 1e-2 normwise bound against the FP64 oracle run on the
    FP32 master weights (features and weights rounded to BF16 on the GPU)."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    seed, depth, V, F = 1301, 5, [17, 17, 9, 9, 5, 3], 8
    tree = A.octree_build(seed, depth, 0.6, V)
    ot = O.build_tree(seed, depth, 0.6, V)
    tables = I.make_tables(seed + 1, tree.num_texels, F, 0.3)
    if tdt == torch.float16:
        tables = tables.astype(np.float16).astype(np.float32)
    weights = I.make_mlp(seed + 2, [(depth + 1) * F, 64, 64, 3])
    sc = A.Scene(tree, dev(tables).to(tdt).contiguous(),
                 [dev(W).to(torch.bfloat16) for W in weights], device=DEV,
                 query_form=L.OCTA_FORM_TRILINEAR_VERTEX)
    x, w = I.uniform_queries(seed + 3, 3001)
    rgb, _, addr = A.octa_query_fwd(sc, dev(x), dev(w), want_addr=True)
    ref, enc = O.query_forward(ot, tables, weights, x, w, form="full")
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr.reshape(len(x), depth + 1, 24))
    err = np.linalg.norm(rgb.cpu().numpy() - ref) / np.linalg.norm(ref)
    print("BF16 full-form forward, normwise error", err)
    assert err <= 1e-2


# ------------------------------------ BF16 tensor-core backward / training

def _mask_fraction(weights, h):
    """Fraction of hidden pre-activations within the BF16 forward error bound
    2^-7 sum |w||a| of zero (their ReLU masks may differ from FP64's)."""
    a = np.asarray(h, np.float64)
    flags = []
    for W in [np.asarray(W, np.float64) for W in weights][:-1]:
        z = a @ W.T
        flags.append((np.abs(z) < 2.0 ** -7 * (np.abs(a) @ np.abs(W).T)).ravel())
        a = np.maximum(z, 0.0)
    return float(np.mean(np.concatenate(flags)))


def test_full_form_bf16_backward_vs_oracle():
    """octa_query_bwd on a BF16 decoder in the full form against the FP64
    oracle on the quantised parameters: the last layer's dW (no ReLU mask)
    to 1e-2, the other tensors to 3 sqrt(f) + 1e-2 with f the fraction of
    pre-activations whose mask BF16 may flip (the bound of the cell form's
    BF16 backward tests)."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    seed, depth, V, F = 1311, 5, [17, 17, 9, 9, 5, 3], 8
    tree = A.octree_build(seed, depth, 0.6, V)
    ot = O.build_tree(seed, depth, 0.6, V)
    tq = I.make_tables(seed + 1, tree.num_texels, F, 0.3).astype(np.float16).astype(np.float32)
    weights = [W * np.float32(1.5) for W in I.make_mlp(seed + 2, [(depth + 1) * F, 64, 64, 3])]
    Wb = [dev(W).to(torch.bfloat16) for W in weights]
    wq = [W.float().cpu().numpy() for W in Wb]
    sc = A.Scene(tree, dev(tq).half().contiguous(), Wb, device=DEV,
                 query_form=L.OCTA_FORM_TRILINEAR_VERTEX)
    x, w = I.uniform_queries(seed + 3, 6000)
    d_rgb = np.random.default_rng(seed).normal(size=(len(x), 3)).astype(np.float32)
    dT = torch.zeros((tree.num_texels, F), device=DEV)
    dW = torch.zeros(sc.weights.shape, device=DEV)
    A.octa_query_bwd(sc, dev(x), dev(w), dev(d_rgb), [(dT, dW)])
    rT, rWs, _ = O.query_backward(ot, tq, wq, x, w, d_rgb, form="full")
    frac = _mask_fraction(wq, O.encode_features_full(ot, tq, x, w).h)
    errs = [_normwise(dT.cpu().numpy(), rT)]
    gw = dW.cpu().numpy()
    for (off, o, i), rW in zip(sc.weight_slices(), rWs):
        errs.append(_normwise(gw[off:off + o * i].reshape(o, i), rW))
    print("BF16 full-form backward errors", [round(e, 5) for e in errs], "mask fraction", frac)
    assert errs[-1] <= 1e-2
    assert max(errs[:-1]) <= 3.0 * np.sqrt(frac) + 1e-2


def test_full_form_bf16_fused_and_one_launch_training():
    """train_bf16's shapes (BF16 decoder, FP16 tables) on vertex maps of side
    R + 1 in the full form, 4,097 pairs: the fused training pass against the
    unfused forward + loss + backward (same arithmetic up to the atomics'
    order), its loss against the FP64 oracle (1e-2), and the one-launch
    step against the fused pass followed by Adam."""
    from paper_2606_08469_gb300 import api as A
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_bf16"]
    a, (tree, tables, weights, pairs) = WL.train_step_for(cfg, n_pairs=4097, query_form="full")
    b, _ = WL.train_step_for(cfg, n_pairs=4097, query_form="full", fused=True)
    a.forward()
    a.loss_and_grad()
    a.backward()
    b.fused_pass()
    torch.cuda.synchronize()
    assert abs(a.loss.item() - b.loss.item()) <= 1e-6 * a.loss.item()
    for sa, sb in zip(a.states, b.states):
        for ga, gb in ((sa.grad_t, sb.grad_t), (sa.grad_w, sb.grad_w)):
            assert (torch.linalg.norm(ga - gb) / torch.linalg.norm(gb)).item() <= 1e-4
    ot = O.build_tree(cfg.seed("tree"), cfg.max_depth, cfg.p_base, [r + 1 for r in cfg.R])
    N = pairs.n
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    rgb, _ = O.query_forward(ot, tables, weights, X, Om, form="full")
    loss, _, _ = O.residual_loss(rgb[:N], rgb[N:], pairs.E, pairs.w)
    assert abs(b.loss.item() - loss) <= 1e-2 * loss
    c, _ = WL.train_step_for(cfg, n_pairs=4097, query_form="full", fused=True)
    d, _ = WL.train_step_for(cfg, n_pairs=4097, query_form="full", persistent=True)
    for _ in range(2):
        c.step()
        d.step()
        torch.cuda.synchronize()
        torch.testing.assert_close(d.loss, c.loss, rtol=1e-6, atol=0)
        sc_, sd_ = A.read_scaler(c.scaler), A.read_scaler(d.scaler)
        assert (sc_.step, sc_.skipped) == (sd_.step, sd_.skipped)


def test_full_form_config3_frame_samples():
    """The full-form legs' configuration at full size: gbuffer_frame's 1280x720
    G-buffer on its depth-8 octree with vertex maps 65 ... 9, FP16 tables.
    On 2,000 sampled queries: the 24 entries of every level bit-exact, the
    BF16 features within BF16 rounding of the oracle's, the tensor-core
    forward within the BF16 path's 1e-2 normwise bound."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    cfg = I.WORKLOADS["gbuffer_frame"]
    V = [r + 1 for r in cfg.R]
    tree = A.octree_build(cfg.seed("tree"), cfg.max_depth, cfg.p_base, V)
    ot = O.build_tree(cfg.seed("tree"), cfg.max_depth, cfg.p_base, V)
    tables = I.make_tables(cfg.seed("tables"), tree.num_texels, cfg.F, cfg.sigma)
    tq = tables.astype(np.float16).astype(np.float32)
    mlp = I.make_mlp(cfg.seed("mlp"), [tree.num_levels * cfg.F, 64, 64, 3])
    sc = A.Scene(tree, dev(tq).half().contiguous(), [dev(W).to(torch.bfloat16) for W in mlp],
                 device=DEV, query_form=L.OCTA_FORM_TRILINEAR_VERTEX)
    x, om = I.gbuffer_queries(cfg.seed("queries"), 1280, 720)
    feat, _, addr = A.octa_encode(sc, dev(x), dev(om), feat_dtype=torch.bfloat16, want_addr=True)
    rgb, _, _ = A.octa_query_fwd(sc, dev(x), dev(om))
    rows = np.random.default_rng(4).choice(len(x), 2000, replace=False)
    ref = O.encode_features_full(ot, tq, x[rows], om[rows])
    K = tree.num_levels
    np.testing.assert_array_equal(addr.cpu().numpy()[rows], ref.addr.reshape(len(rows), K, 24))
    np.testing.assert_allclose(feat.float().cpu().numpy()[rows], ref.h, rtol=2 ** -8,
                               atol=64 * U32 * np.abs(tq).max())
    r_ref, _ = O.query_forward(ot, tq, mlp, x[rows], om[rows], form="full")
    got = rgb.cpu().numpy()[rows]
    assert np.linalg.norm(got - r_ref) <= 1e-2 * np.linalg.norm(r_ref)
