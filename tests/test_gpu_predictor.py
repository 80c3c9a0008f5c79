"""The disparity predictor g_psi (octa_disparity) against the FP64 oracle,
and the inference path predictor -> disparity-shifted encoding (Eq. 7-9)
end to end."""
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


def _predictor(seed, levels, log2_T, n_min, n_max, wscale=1.0):
    g = I.rng(seed)
    res = O.hash_resolutions(levels, n_min, n_max)
    table = g.uniform(-1e-1, 1e-1, (levels, 1 << log2_T, 2)).astype(np.float32)
    weights = [W * np.float32(wscale) for W in I.make_mlp(seed + 1, [2 * levels + 3, 64, 64, 1])]
    return table, res, weights


def _queries(seed, n):
    g = I.rng(seed)
    x = g.random((n, 3)).astype(np.float32)
    w = I.unit_vectors(g, n).astype(np.float32)
    nrm = (I.unit_vectors(g, n) * g.uniform(0.5, 2, (n, 1))).astype(np.float32)
    x[:5] = np.float32(1.0)                       # the cube's far corner (cell clamp)
    return x, w, nrm


@pytest.mark.parametrize("levels,log2_T,n_min,n_max,wscale", [
    (8, 16, 16, 512, 1.0),     # the first levels dense, the rest hashed
    (4, 14, 2, 8, 3.0),        # all dense
    (16, 12, 16, 4096, 1.0),   # hashed, many collisions, the widest input
])
def test_disparity_matches_oracle(levels, log2_T, n_min, n_max, wscale):
    """FP32 against FP64: |d_gpu / d - 1| = |dz| <= max(1e-5, 16 u z_abs),
    z_abs the MLP run on |W| and |input| (the decoder's bound)."""
    from paper_2606_08469_gb300 import api as A
    table, res, weights = _predictor(600 + levels, levels, log2_T, n_min, n_max, wscale)
    x, w, nrm = _queries(700 + levels, 20001)
    pred = A.Predictor(table, res, weights, device=DEV)
    d = A.octa_disparity(pred, dev(x), dev(w), dev(nrm)).cpu().numpy()
    ref = O.disparity(table, res, weights, x, w, nrm)
    inp = np.concatenate([O.hash_encode(table, res, x),
                          O.reflect_f32(w, nrm).astype(np.float64)], axis=1)
    _, zs, _ = O.mlp_forward([np.abs(W) for W in weights], np.abs(inp))
    tol = np.maximum(1e-5, 16 * U32 * zs[-1][:, 0])
    err = np.abs(d / ref - 1)
    assert np.all(err <= tol), (err.max(), tol.min())


def test_predictor_then_shifted_encoding():
    """Inference path: octa_disparity feeds octa_encode in the shifted form;
    with the GPU's disparities the 24 entries of every level are the
    oracle's bit for bit and the features within the binary32 bound."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    table, res, weights = _predictor(800, 8, 16, 16, 512)
    pred = A.Predictor(table, res, weights, device=DEV)
    V = [17, 17, 9, 9, 5, 3]
    tree = A.octree_build(801, 5, 0.6, V)
    ot = O.build_tree(801, 5, 0.6, V)
    tables = I.make_tables(802, tree.num_texels, 8, 0.3)
    sc = A.Scene(tree, dev(tables), [dev(W) for W in I.make_mlp(803, [48, 16, 3])], device=DEV,
                 query_form=L.OCTA_FORM_SHIFTED)
    x, w, nrm = _queries(804, 5000)
    X, Wd, Nd = dev(x), dev(w), dev(nrm)
    d = A.octa_disparity(pred, X, Wd, Nd)
    feat, _, addr = A.octa_encode(sc, X, Wd, want_addr=True, normal=Nd, disparity=d)
    ref = O.encode_features_shifted(ot, tables, x, w, nrm, d.cpu().numpy())
    np.testing.assert_array_equal(addr.cpu().numpy(), ref.addr.reshape(len(x), 6, 24))
    np.testing.assert_allclose(feat.cpu().numpy(), ref.h, rtol=1e-6, atol=64 * U32 * 1.5)


def test_predictor_errors():
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    table, res, weights = _predictor(900, 2, 8, 4, 8)
    pred = A.Predictor(table, res, weights, device=DEV)
    x, w, nrm = _queries(901, 10)
    with pytest.raises(L.OctaError):
        q = A._queries(dev(x), dev(w), None)      # no normal
        L.check(A._lib().octa_disparity(A.C.byref(pred.as_c()), A.C.byref(q),
                                        A._ptr(torch.empty(10, device=DEV)), A._stream()), "d")
    bad = pred.as_c()
    bad.levels = 17
    with pytest.raises(L.OctaError):
        q = A._queries(dev(x), dev(w), None)
        q.normal = dev(nrm).data_ptr()
        L.check(A._lib().octa_disparity(A.C.byref(bad), A.C.byref(q),
                                        A._ptr(torch.empty(10, device=DEV)), A._stream()), "d")
    assert A.octa_disparity(pred, dev(x)[:0], dev(w)[:0], dev(nrm)[:0]).numel() == 0


def _attrs(x, w, nrm, seed):
    """Eq. 12's g: position, reflection direction, normal, albedo, roughness."""
    g = I.rng(seed)
    n = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    return np.concatenate([x, O.reflect_f32(w, nrm), n, g.random((len(x), 3)),
                           g.uniform(0.05, 0.6, (len(x), 1))], axis=1).astype(np.float32)


def test_full_inference_path_tensor_cores():
    """The paper's inference: d = g_psi(x, omega_r) (octa_disparity), then
    octa_query_fwd in the shifted form on a BF16 decoder whose input is
    [h, g] (K F = 72 features + 13 attributes, the 96-wide operand): the 24
    entries of every level bit-exact given the GPU's d, radiance within the
    BF16 path's 1e-2 normwise bound against the FP64 oracle."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    table, res, pw = _predictor(1000, 8, 16, 16, 512)
    pred = A.Predictor(table, res, pw, device=DEV)
    V = [65, 65, 33, 33, 17, 17, 9, 9, 9]
    tree = A.octree_build(1001, 8, 0.6, V)
    ot = O.build_tree(1001, 8, 0.6, V)
    tables = I.make_tables(1002, tree.num_texels, 8, 0.3).astype(np.float16).astype(np.float32)
    weights = I.make_mlp(1003, [72 + 13, 64, 64, 3])
    sc = A.Scene(tree, dev(tables).half().contiguous(), [dev(W).to(torch.bfloat16) for W in weights],
                 device=DEV, query_form=L.OCTA_FORM_SHIFTED)
    x, w, nrm = _queries(1004, 3001)
    g = _attrs(x, w, nrm, 1005)
    X, Wd, Nd, G = dev(x), dev(w), dev(nrm), dev(g)
    d = A.octa_disparity(pred, X, Wd, Nd)
    rgb, _, addr = A.octa_query_fwd(sc, X, Wd, want_addr=True, normal=Nd, disparity=d, attrs=G)
    dd = d.cpu().numpy()
    ref, enc = O.query_forward(ot, tables, weights, x, w, form="shifted", normal=nrm,
                               disparity=dd, attrs=g)
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr.reshape(len(x), 9, 24))
    err = np.linalg.norm(rgb.cpu().numpy() - ref) / np.linalg.norm(ref)
    print("full inference path, BF16 normwise error", err)
    assert err <= 1e-2


def test_attributes_fp32_forward_and_backward():
    """Eq. 12 on the FP32 engine (cell form, K F = 56 + 13 attributes in the
    72-wide shape): radiance to 1e-5 and table / weight gradients (the
    attributes' W1 columns included) to 1e-5 normwise against the oracle."""
    from paper_2606_08469_gb300 import api as A
    cfg = I.WORKLOADS["train_f32"]
    tree = A.octree_build(cfg.seed("tree"), cfg.max_depth, cfg.p_base, cfg.R)
    ot = O.build_tree(cfg.seed("tree"), cfg.max_depth, cfg.p_base, cfg.R)
    tables = I.make_tables(1101, tree.num_texels, 8, 0.3)
    weights = I.make_mlp(1102, [56 + 13, 64, 64, 3])
    sc = A.Scene(tree, dev(tables), [dev(W) for W in weights], device=DEV)
    x, w, nrm = _queries(1103, 4097)
    g = _attrs(x, w, nrm, 1104)
    rgb, _, _ = A.octa_query_fwd(sc, dev(x), dev(w), attrs=dev(g))
    ref, _ = O.query_forward(ot, tables, weights, x, w, attrs=g)
    assert np.max(np.abs(rgb.cpu().numpy() / ref - 1)) <= 1e-5
    d_rgb = np.random.default_rng(5).normal(size=(len(x), 3)).astype(np.float32)
    dT = torch.zeros((tree.num_texels, 8), device=DEV)
    dW = torch.zeros(sc.weights.shape, device=DEV)
    A.octa_query_bwd(sc, dev(x), dev(w), dev(d_rgb), [(dT, dW)], attrs=dev(g))
    rT, rWs, _ = O.query_backward(ot, tables, weights, x, w, d_rgb, attrs=g)
    assert np.linalg.norm(dT.cpu().numpy() - rT) <= 1e-5 * np.linalg.norm(rT)
    gw = dW.cpu().numpy()
    for (off, o, i), rW in zip(sc.weight_slices(), rWs):
        assert np.linalg.norm(gw[off:off + o * i].reshape(o, i) - rW) <= 1e-5 * np.linalg.norm(rW)


@pytest.mark.parametrize("levels,log2_T", [(8, 16), (14, 12)])
def test_disparity_tensor_cores(levels, log2_T):
    """g_psi's MLP on the tcgen05 path (BF16 inputs and weights, FP32
    accumulation) against the FP64 oracle on the FP32 master weights: the
    BF16 path's 1e-2 normwise bound, and per query |d / d_ref - 1| = |dz|
    within the BF16 rounding of inputs and weights, 2^-6 z_abs + 1e-3 (z_abs
    the MLP on |W| and |input|); the ragged tail of a 20,001-query batch
    included."""
    from paper_2606_08469_gb300 import api as A
    table, res, weights = _predictor(640 + levels, levels, log2_T, 16, 512)
    x, w, nrm = _queries(740 + levels, 20001)
    pred = A.Predictor(table, res, weights, device=DEV, tensor_cores=True)
    d = A.octa_disparity(pred, dev(x), dev(w), dev(nrm)).cpu().numpy()
    ref = O.disparity(table, res, weights, x, w, nrm)
    inp = np.concatenate([O.hash_encode(table, res, x),
                          O.reflect_f32(w, nrm).astype(np.float64)], axis=1)
    _, zs, _ = O.mlp_forward([np.abs(W) for W in weights], np.abs(inp))
    err = np.abs(d / ref - 1)
    tol = 2.0 ** -6 * zs[-1][:, 0] + 1e-3
    print("tensor-core predictor: max |d/d_ref - 1|", err.max(), "median tol", np.median(tol))
    assert np.all(err <= tol)
    assert np.linalg.norm(d - ref) <= 1e-2 * np.linalg.norm(ref)   # the BF16 path's binding bound
