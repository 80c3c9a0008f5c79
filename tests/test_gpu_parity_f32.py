"""GPU parity of the FP32 path against the FP64 oracle (through the C ABI).

Node indices and texel addresses must agree bit for bit; FP32 radiance to
1e-5 relative (elementwise; radiance = exp(.) > 0); FP32 gradients to 1e-5
normwise per parameter tensor.  The oracle always works on its own tree,
rebuilt from the seed, never on the library's output."""
import numpy as np
import pytest
import torch

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda"
RTOL_RGB = 1e-5
RTOL_GRAD = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_08469_gb300 import build
    build.build()


def api():
    from paper_2606_08469_gb300 import api as A
    return A


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def oracle_tree(seed, depth, R, p=0.6):
    return O.build_tree(seed, depth, p, R)


def make_scene(seed, depth, R, F, sigma, widths_hidden, tdt=torch.float32, wscale=1.0,
               tseed=2000, wseed=3000):
    A = api()
    tree = A.octree_build(seed, depth, 0.6, R)
    tables = I.make_tables(tseed, tree.num_texels, F, sigma)
    weights = [W * np.float32(wscale) for W in I.make_mlp(wseed, [(depth + 1) * F] + widths_hidden + [3])]
    if tdt == torch.float16:
        tables = tables.astype(np.float16).astype(np.float32)   # the values the GPU reads
    sc = A.Scene(tree, dev(tables).to(tdt).contiguous(), [dev(W) for W in weights], device=DEV)
    return sc, oracle_tree(seed, depth, R), tables, weights


def rel_err(a, b):
    return np.max(np.abs(a - b) / np.abs(b))


U32 = 2.0 ** -24


def rgb_tolerance(weights, h):
    """Per-element bound on |rgb_gpu / rgb - 1| for an FP32 evaluation.

    The relative error of exp(z) equals the absolute error of z.  FP32 dot
    products of n terms carry |dz| <= gamma_n sum |w||a|; propagated through
    the layers this is bounded by c * u * z_abs, with z_abs the output of the
    same network run on |W| and |h| (ReLU is the identity there).  c = 16 is
    a statistical (sqrt n) rather than worst-case constant.  The 1e-5 floor
    is the stated FP32 tolerance, which the configurations' own inputs meet.
    """
    _, zs, _ = O.mlp_forward([np.abs(W) for W in weights], np.abs(h))
    return np.maximum(1e-5, 16 * U32 * zs[-1])


def assert_rgb(gpu, ref, weights, h):
    err = np.abs(gpu - ref) / ref
    tol = rgb_tolerance(weights, h)
    assert np.all(err <= tol), (err.max(), tol[np.unravel_index(np.argmax(err / tol), err.shape)])


def normwise(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------ forward

@pytest.mark.parametrize("sigma,wscale", [(0.1, 1.0), (0.6, 3.0)])
def test_forward_config0_full(sigma, wscale):
    """16384 queries, depth-4 tree, R = 16,16,8,8,8, F = 4, 20-32-32-3."""
    cfg = I.WORKLOADS["forward_small"]
    sc, ot, tables, weights = make_scene(cfg.seed("tree"), 4, cfg.R, 4, sigma, [32, 32],
                                         wscale=wscale, tseed=cfg.seed("tables"),
                                         wseed=cfg.seed("mlp"))
    x, w = I.uniform_queries(cfg.seed("queries"), cfg.n)
    rgb, nodes, addr = api().octa_query_fwd(sc, dev(x), dev(w), want_nodes=True, want_addr=True)
    ref, enc = O.query_forward(ot, tables, weights, x, w)
    np.testing.assert_array_equal(nodes.cpu().numpy(), enc.node)
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr)
    if wscale == 1.0:
        assert rel_err(rgb.cpu().numpy(), ref) <= RTOL_RGB     # the workload's own inputs
    else:
        assert ref.max() / ref.min() > 5          # the test exercises the nonlinearity
        assert_rgb(rgb.cpu().numpy(), ref, weights, enc.h)


def test_encode_features_match_oracle():
    cfg = I.WORKLOADS["train_f32"]
    sc, ot, tables, weights = make_scene(cfg.seed("tree"), 6, cfg.R, 8, 0.3, [64, 64])
    pairs = I.training_pairs(cfg.seed("queries"), 5000)
    feat, nodes, addr = api().octa_encode(sc, dev(pairs.x), dev(pairs.omega), want_nodes=True,
                                          want_addr=True)
    enc = O.encode_features(ot, tables, pairs.x, pairs.omega)
    np.testing.assert_array_equal(nodes.cpu().numpy(), enc.node)
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr)
    np.testing.assert_allclose(feat.cpu().numpy(), enc.h, rtol=1e-5, atol=2e-6)
    fb, _, _ = api().octa_encode(sc, dev(pairs.x), dev(pairs.omega), feat_dtype=torch.bfloat16)
    np.testing.assert_allclose(fb.float().cpu().numpy(), enc.h, rtol=1e-2, atol=1e-3)


def test_encode_two_scenes_strided_rows():
    """Scenes with K*F = 40 and 56 in one call: rows of the shallower scene
    are shorter than the row stride (strided copy-out), its tail untouched."""
    A = api()
    parts = []
    for s, (seed, depth) in enumerate([(1400, 4), (1402, 6)]):
        R = I.R_DEEP[:depth + 1]
        tree = A.octree_build(seed, depth, 0.6, R)
        tables = I.make_tables(2400 + s, tree.num_texels, 8, 0.3)
        weights = I.make_mlp(3400 + s, [(depth + 1) * 8, 64, 64, 3])
        parts.append((A.Scene(tree, dev(tables), [dev(W) for W in weights], device=DEV),
                      O.build_tree(seed, depth, 0.6, R), tables))
    counts = [333, 1000]
    xs, ws = zip(*[I.uniform_queries(70 + s, n) for s, n in enumerate(counts)])
    # FP32: the texel coordinate p = uv R - 1/2 carries ~u R of rounding and h
    # moves by at most 2 max|T| per unit of p: |dh| <= 4 u R_max max|T|
    tmax = max(float(np.abs(p[2]).max()) for p in parts)
    atol32 = 4 * 2.0 ** -24 * 64 * tmax
    for dt, rtol, atol in ((torch.float32, 1e-5, atol32), (torch.bfloat16, 1e-2, 1e-3)):
        feat, nodes, addr = A.octa_encode([p[0] for p in parts], dev(np.concatenate(xs)),
                                          dev(np.concatenate(ws)), counts, feat_dtype=dt,
                                          want_nodes=True, want_addr=True)
        f = feat.float().cpu().numpy()
        off = 0
        for s, n in enumerate(counts):
            enc = O.encode_features(parts[s][1], parts[s][2], xs[s], ws[s])
            W = enc.h.shape[1]
            np.testing.assert_allclose(f[off:off + n, :W], enc.h, rtol=rtol, atol=atol)
            assert not f[off:off + n, W:].any()
            K = parts[s][1].num_levels
            np.testing.assert_array_equal(addr.cpu().numpy()[off:off + n, :K], enc.addr)
            off += n


def _edge_queries():
    s = 1.0 / np.sqrt(2.0)
    w = np.array([[0, 0, 1], [0, 0, -1], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0],
                  [s, s, 0], [s, 0, -s], [0, -s, -s], [-0.0, 0.5, -0.5], [0.5, -0.0, -0.5],
                  [1e-30, 1, 1e-30], [0.3, 0.4, -1e-7], [0.3, 0.4, 1e-7]], dtype=np.float32)
    x = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5], [0.25, 0.75, 1.0], [1.0, 0, 0.5],
                  [0.999999, 0.5, 0.0], [0.0625, 0.125, 0.1875], [-0.5, 1.5, 0.5],
                  [0.5, 0.5, 0.5], [0.1, 0.9, 0.3], [0.7, 0.2, 0.4], [0.3, 0.3, 0.3],
                  [0.8, 0.8, 0.8], [0.8, 0.8, 0.8]], dtype=np.float32)
    return x, w


@pytest.mark.parametrize("n", [1, 127, 129, 300, 4097])
def test_forward_ragged_and_edges(n):
    cfg = I.WORKLOADS["train_f32"]
    sc, ot, tables, weights = make_scene(cfg.seed("tree"), 6, cfg.R, 8, 0.3, [64, 64], wscale=2.0)
    xe, we = _edge_queries()
    x, w = I.uniform_queries(77 + n, n)
    k = min(n, len(xe))
    x[:k], w[:k] = xe[:k], we[:k]
    rgb, nodes, addr = api().octa_query_fwd(sc, dev(x), dev(w), want_nodes=True, want_addr=True)
    ref, enc = O.query_forward(ot, tables, weights, x, w)
    np.testing.assert_array_equal(nodes.cpu().numpy(), enc.node)
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr)
    assert_rgb(rgb.cpu().numpy(), ref, weights, enc.h)


def test_forward_empty_batch_is_a_no_op():
    cfg = I.WORKLOADS["forward_small"]
    sc, _, _, _ = make_scene(cfg.seed("tree"), 4, cfg.R, 4, 0.1, [32, 32])
    x = torch.empty((0, 3), device=DEV)
    rgb, _, _ = api().octa_query_fwd(sc, x, x)
    assert rgb.shape == (0, 3)


def test_forward_hand_tree_absent_levels():
    """A tree that splits only one octant: most queries have absent deep
    levels (address -1, zero features)."""
    A = api()
    flags = [1, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 1]
    R = [8, 4, 4, 2]
    tree = A.octree_from_flags(flags, 3, R)
    ot = O.tree_from_flags(flags, 3, R)
    tables = I.make_tables(5, tree.num_texels, 4, 0.5)
    weights = I.make_mlp(6, [16, 32, 32, 3])
    sc = A.Scene(tree, dev(tables), [dev(W) for W in weights], device=DEV)
    x, w = I.uniform_queries(9, 3000)
    rgb, nodes, addr = A.octa_query_fwd(sc, dev(x), dev(w), want_nodes=True, want_addr=True)
    ref, enc = O.query_forward(ot, tables, weights, x, w)
    assert (enc.node[:, 3] >= 0).mean() < 0.1 and (enc.node[:, 3] >= 0).any()
    np.testing.assert_array_equal(nodes.cpu().numpy(), enc.node)
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr)
    assert_rgb(rgb.cpu().numpy(), ref, weights, enc.h)


def test_forward_fp16_tables_fp32_decoder():
    cfg = I.WORKLOADS["train_bf16"]
    sc, ot, tables, weights = make_scene(cfg.seed("tree"), 8, cfg.R, 8, 0.3, [64, 64, 64],
                                         tdt=torch.float16, wscale=2.0)
    x, w = I.uniform_queries(21, 6000)
    rgb, nodes, addr = api().octa_query_fwd(sc, dev(x), dev(w), want_nodes=True, want_addr=True)
    ref, enc = O.query_forward(ot, tables, weights, x, w)
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr)
    assert_rgb(rgb.cpu().numpy(), ref, weights, enc.h)


def test_malformed_tree_reports_status():
    """Child / map ranges outside the arrays are flagged, never read."""
    A = api()
    tree = A.octree_build(3, 2, 1.0, [4, 4, 4])
    tables = I.make_tables(1, tree.num_texels, 4, 0.1)
    weights = I.make_mlp(2, [12, 32, 32, 3])
    fc = tree.first_child.copy()
    fc[0] = tree.num_nodes - 3          # children would run past the node array
    tree.first_child[:] = fc
    sc = A.Scene(tree, dev(tables), [dev(W) for W in weights], device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    x, w = I.uniform_queries(4, 500)
    rgb, nodes, _ = A.octa_query_fwd(sc, dev(x), dev(w), want_nodes=True, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & 1
    assert torch.isfinite(rgb).all() and (nodes[:, 1:] == -1).all()
    mo = tree.map_offset.copy()
    mo[0] = tree.num_texels - 2         # root map would run past the table
    tree.map_offset[:] = mo
    tree.first_child[:] = -1
    sc2 = A.Scene(tree, dev(tables), [dev(W) for W in weights], device=DEV)
    status.zero_()
    A.octa_query_fwd(sc2, dev(x), dev(w), status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & 2



@pytest.mark.parametrize("form", ["cell", "full"])
@pytest.mark.parametrize("bad", [-1, -16])
def test_negative_map_offset_reports_status(form, bad):
    """A map base before the table start (negative offset, including ones
    whose unsigned sum with R^2 lands back inside the table) is flagged as
    OCTA_STATUS_BAD_MAP and never read: the encoding (shared gather) and the
    FP32 engine's forward both treat the level as absent."""
    from paper_2606_08469_gb300 import _lib as L
    A = api()
    R = [4, 4, 4] if form == "cell" else [5, 5, 5]
    qf = L.OCTA_FORM_CELL_BILINEAR if form == "cell" else L.OCTA_FORM_TRILINEAR_VERTEX
    tree = A.octree_build(3, 2, 1.0, R)
    tables = I.make_tables(1, tree.num_texels, 4, 0.1)
    weights = I.make_mlp(2, [12, 32, 32, 3])
    tree.map_offset[:] = tree.map_offset.copy()
    tree.map_offset[0] = bad          # the root's map would start before the table
    sc = A.Scene(tree, dev(tables), [dev(W) for W in weights], device=DEV, query_form=qf)
    x, w = I.uniform_queries(4, 500)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    feat, _, _ = A.octa_encode(sc, dev(x), dev(w), status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & 2
    assert torch.isfinite(feat).all() and (feat[:, :4] == 0).all()   # level 0 absent
    status.zero_()
    rgb, _, _ = A.octa_query_fwd(sc, dev(x), dev(w), status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & 2
    assert torch.isfinite(rgb).all()

# ----------------------------------------------------------------- backward

@pytest.mark.parametrize("which", ["forward_small", "train_f32"])
def test_backward_matches_oracle(which):
    cfg = I.WORKLOADS[which]
    hidden = [32, 32] if which == "forward_small" else [64, 64]
    sc, ot, tables, weights = make_scene(cfg.seed("tree"), cfg.max_depth, cfg.R, cfg.F, 0.3,
                                         hidden, wscale=1.5)
    x, w = I.uniform_queries(31 + cfg.index, 12000)
    d_rgb = np.random.default_rng(5).normal(size=(len(x), 3)).astype(np.float32)
    dT = torch.zeros(sc.tables.shape, device=DEV)
    dW = torch.zeros(sc.weights.shape, device=DEV)
    api().octa_query_bwd(sc, dev(x), dev(w), dev(d_rgb), [(dT, dW)])
    rT, rWs, _ = O.query_backward(ot, tables, weights, x, w, d_rgb)
    assert normwise(dT.cpu().numpy(), rT) <= RTOL_GRAD
    gw = dW.cpu().numpy()
    for (off, o, i), rW in zip(sc.weight_slices(), rWs):
        assert normwise(gw[off:off + o * i].reshape(o, i), rW) <= RTOL_GRAD


def test_backward_fd_subset_config1():
    """GPU gradient of the Eq. 14 loss on 64 pairs of the config-1 workload vs
    central differences (FP64 oracle) of the frozen-normaliser surrogate."""
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_f32"]
    step, (tree, tables, weights, pairs) = WL.train_step_for(cfg, n_pairs=64, scale=1.0,
                                                             growth_interval=0)
    step.forward()
    step.loss_and_grad()
    step.backward()
    torch.cuda.synchronize()
    gT = step.states[0].grad_t.cpu().numpy().astype(np.float64)
    gW = step.states[0].grad_w.cpu().numpy().astype(np.float64)
    ot = oracle_tree(cfg.seed("tree"), cfg.max_depth, cfg.R)
    N = pairs.n
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    rgb, _ = O.query_forward(ot, tables, weights, X, Om)
    T0 = pairs.E + pairs.w * rgb[N:]
    D0 = rgb[:N] + T0

    def Lsur(T_, Ws_):
        return O.surrogate_loss(ot, T_, Ws_, pairs.x, pairs.omega, pairs.x2, -pairs.omega2,
                                pairs.E, pairs.w, D0, T0, 1e-2, True)
    g = np.random.default_rng(3)
    T64 = tables.astype(np.float64)
    W64 = [W.astype(np.float64) for W in weights]
    touched = np.nonzero(np.abs(gT).sum(1) > 0)[0]
    h = 1e-6
    for r in g.choice(touched, 12, replace=False):
        f = int(g.integers(0, cfg.F))
        Tp, Tm = T64.copy(), T64.copy()
        Tp[r, f] += h
        Tm[r, f] -= h
        fd = (Lsur(Tp, W64) - Lsur(Tm, W64)) / (2 * h)
        assert abs(gT[r, f] - fd) <= 1e-3 * abs(fd) + 1e-9, (r, f, gT[r, f], fd)
    off = 0
    for li, W in enumerate(W64):
        for _ in range(6):
            i, j = int(g.integers(0, W.shape[0])), int(g.integers(0, W.shape[1]))
            Wp = [w.copy() for w in W64]
            Wm = [w.copy() for w in W64]
            Wp[li][i, j] += h
            Wm[li][i, j] -= h
            fd = (Lsur(T64, Wp) - Lsur(T64, Wm)) / (2 * h)
            an = gW[off + i * W.shape[1] + j]
            assert abs(an - fd) <= 1e-3 * abs(fd) + 1e-9, (li, i, j, an, fd)
        off += W.size


def test_batched_scenes_match_oracle():
    """Three trees of different depth, uneven query counts, one launch each
    for forward and backward."""
    A = api()
    specs = [(1400, 4), (1402, 6), (1404, 8)]
    counts = [1000, 5000, 301]
    scenes, otrees, tabs, wts, xs, ws = [], [], [], [], [], []
    for s, ((seed, depth), n) in enumerate(zip(specs, counts)):
        R = I.R_DEEP[:depth + 1]
        sc, ot, t, wt = make_scene(seed, depth, R, 8, 0.3, [64, 64], wscale=1.5, tseed=2400 + s,
                                   wseed=3400 + s)
        x, w = I.uniform_queries(4400 + s, n)
        scenes.append(sc); otrees.append(ot); tabs.append(t); wts.append(wt); xs.append(x); ws.append(w)
    X, W = np.concatenate(xs), np.concatenate(ws)
    rgb, nodes, addr = A.octa_query_fwd(scenes, dev(X), dev(W), counts, want_nodes=True,
                                        want_addr=True)
    d_rgb = np.random.default_rng(8).normal(size=(len(X), 3)).astype(np.float32)
    grads = [(torch.zeros(s.tables.shape, device=DEV), torch.zeros(s.weights.shape, device=DEV))
             for s in scenes]
    A.octa_query_bwd(scenes, dev(X), dev(W), dev(d_rgb), grads, counts)
    rgb = rgb.cpu().numpy()
    nodes = nodes.cpu().numpy()
    off = 0
    for s, n in enumerate(counts):
        sl = slice(off, off + n)
        ref, enc = O.query_forward(otrees[s], tabs[s], wts[s], xs[s], ws[s])
        K = otrees[s].num_levels
        np.testing.assert_array_equal(nodes[sl, :K], enc.node)
        assert (nodes[sl, K:] == -1).all()
        np.testing.assert_array_equal(addr.cpu().numpy()[sl, :K], enc.addr)
        assert_rgb(rgb[sl], ref, wts[s], enc.h)
        rT, rWs, _ = O.query_backward(otrees[s], tabs[s], wts[s], xs[s], ws[s], d_rgb[sl])
        assert normwise(grads[s][0].cpu().numpy(), rT) <= RTOL_GRAD
        gw = grads[s][1].cpu().numpy()
        for (o_, a, b), rW in zip(scenes[s].weight_slices(), rWs):
            assert normwise(gw[o_:o_ + a * b].reshape(a, b), rW) <= RTOL_GRAD
        off += n


def test_autograd_function():
    A = api()
    cfg = I.WORKLOADS["forward_small"]
    sc, ot, tables, weights = make_scene(cfg.seed("tree"), 4, cfg.R, 4, 0.3, [32, 32])
    x, w = I.uniform_queries(55, 2048)
    T = sc.tables.clone().requires_grad_(True)
    Wf = sc.weights.clone().requires_grad_(True)
    rgb = A.octa_query(sc, dev(x), dev(w), T, Wf)
    c = torch.from_numpy(np.random.default_rng(1).normal(size=(len(x), 3)).astype(np.float32)).to(DEV)
    (rgb * c).sum().backward()
    rT, rWs, _ = O.query_backward(ot, tables, weights, x, w, c.cpu().numpy())
    assert normwise(T.grad.cpu().numpy(), rT) <= RTOL_GRAD
    assert normwise(Wf.grad.cpu().numpy(), np.concatenate([r.reshape(-1) for r in rWs])) <= RTOL_GRAD
