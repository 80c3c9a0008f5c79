"""The disparity-shifted lookup (OCTA_FORM_SHIFTED: Eq. 7-9 with Eq. 10 and
Eq. 6) in octa_encode against the FP64 oracle: the 24 vertex entries of every
level bit-exact (the reflection, the per-cell direction, the fold and the
triangle decided in binary32 in the same order on both sides), the features
within the binary32 bound of a 24-term blend."""
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


def _case(seed, depth, V, F, n, tdt=torch.float32, dmax=10.0):
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    tree = A.octree_build(seed, depth, 0.6, V)
    ot = O.build_tree(seed, depth, 0.6, V)
    tables = I.make_tables(seed + 1, tree.num_texels, F, 0.3)
    if tdt == torch.float16:
        tables = tables.astype(np.float16).astype(np.float32)
    weights = [dev(W) for W in I.make_mlp(seed + 2, [(depth + 1) * F, 16, 3])]
    sc = A.Scene(tree, dev(tables).to(tdt).contiguous(), weights, device=DEV,
                 query_form=L.OCTA_FORM_SHIFTED)
    g = I.rng(seed + 3)
    x = g.random((n, 3)).astype(np.float32)
    w = I.unit_vectors(g, n).astype(np.float32)
    nrm = (I.unit_vectors(g, n) * g.uniform(0.5, 2.0, (n, 1))).astype(np.float32)
    d = g.uniform(0.0, dmax, n).astype(np.float32)
    d[:7] = 0.0                                   # the unshifted limit
    return sc, ot, tables, x, w, nrm, d


@pytest.mark.parametrize("seed,depth,V,F,tdt", [
    (1400, 4, [9, 9, 5, 5, 3], 4, torch.float32),
    (1401, 6, [17, 17, 9, 9, 5, 5, 3], 8, torch.float16),
    (1402, 2, [3, 5, 9], 8, torch.float32),
])
def test_shifted_encoding_matches_oracle(seed, depth, V, F, tdt):
    from paper_2606_08469_gb300 import api as A
    sc, ot, tables, x, w, nrm, d = _case(seed, depth, V, F, 4001, tdt)
    feat, _, addr = A.octa_encode(sc, dev(x), dev(w), want_addr=True, normal=dev(nrm),
                                  disparity=dev(d))
    ref = O.encode_features_shifted(ot, tables, x, w, nrm, d)
    np.testing.assert_array_equal(addr.cpu().numpy(), ref.addr.reshape(len(x), depth + 1, 24))
    bound = 64 * U32 * np.abs(tables).max()
    np.testing.assert_allclose(feat.cpu().numpy(), ref.h, rtol=1e-6, atol=bound)


def test_shifted_global_walk_and_errors():
    """A tree larger than the staged capacity; missing inputs are refused, so
    are the FP32 engine's F = 4 shapes (the shifted form is built for F = 8)
    and the one-launch step."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    V = [3, 3, 3, 3, 3]
    tree = A.octree_build(5, 4, 1.0, V)
    assert tree.num_nodes > 2048
    ot = O.build_tree(5, 4, 1.0, V)
    tables = I.make_tables(6, tree.num_texels, 4, 0.3)
    sc = A.Scene(tree, dev(tables), [dev(W) for W in I.make_mlp(7, [20, 32, 32, 3])], device=DEV,
                 query_form=L.OCTA_FORM_SHIFTED)
    g = I.rng(8)
    x = g.random((2000, 3)).astype(np.float32)
    w = I.unit_vectors(g, 2000).astype(np.float32)
    nrm = I.unit_vectors(g, 2000).astype(np.float32)
    d = g.uniform(0, 5, 2000).astype(np.float32)
    feat, _, addr = A.octa_encode(sc, dev(x), dev(w), want_addr=True, normal=dev(nrm),
                                  disparity=dev(d))
    ref = O.encode_features_shifted(ot, tables, x, w, nrm, d)
    np.testing.assert_array_equal(addr.cpu().numpy(), ref.addr.reshape(2000, 5, 24))
    np.testing.assert_allclose(feat.cpu().numpy(), ref.h, rtol=1e-6, atol=64 * U32 * 2.5)
    with pytest.raises(L.OctaError):
        A.octa_encode(sc, dev(x), dev(w))                        # no normal / disparity
    with pytest.raises(L.OctaError):
        A.octa_query_fwd(sc, dev(x), dev(w))                     # no normal / disparity
    with pytest.raises(L.OctaError) as e:                        # FP32 engine, F = 4
        A.octa_query_fwd(sc, dev(x), dev(w), normal=dev(nrm), disparity=dev(d))
    assert e.value.code == L.OCTA_EUNSUPPORTED


def test_shifted_bf16_backward_vs_oracle():
    """octa_query_bwd in the shifted form on a BF16 decoder (the disparity
    given, no gradient to it): table and weight gradients against the FP64
    oracle on the quantised parameters with the BF16 path's ReLU-mask bound
    (the last layer's dW to 1e-2, the rest to 3 sqrt(f) + 1e-2)."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    seed, depth, V, F = 1450, 5, [17, 17, 9, 9, 5, 3], 8
    tree = A.octree_build(seed, depth, 0.6, V)
    ot = O.build_tree(seed, depth, 0.6, V)
    tq = I.make_tables(seed + 1, tree.num_texels, F, 0.3).astype(np.float16).astype(np.float32)
    weights = [W * np.float32(1.5) for W in I.make_mlp(seed + 2, [(depth + 1) * F, 64, 64, 3])]
    Wb = [dev(W).to(torch.bfloat16) for W in weights]
    wq = [W.float().cpu().numpy() for W in Wb]
    sc = A.Scene(tree, dev(tq).half().contiguous(), Wb, device=DEV, query_form=L.OCTA_FORM_SHIFTED)
    g = I.rng(seed + 3)
    n = 6000
    x = g.random((n, 3)).astype(np.float32)
    w = I.unit_vectors(g, n).astype(np.float32)
    nrm = I.unit_vectors(g, n).astype(np.float32)
    d = g.uniform(0, 8, n).astype(np.float32)
    d_rgb = g.normal(size=(n, 3)).astype(np.float32)
    dT = torch.zeros((tree.num_texels, F), device=DEV)
    dW = torch.zeros(sc.weights.shape, device=DEV)
    A.octa_query_bwd(sc, dev(x), dev(w), dev(d_rgb), [(dT, dW)], normal=dev(nrm), disparity=dev(d))
    rT, rWs, _ = O.query_backward(ot, tq, wq, x, w, d_rgb, form="shifted", normal=nrm, disparity=d)
    h = O.encode_features_shifted(ot, tq, x, w, nrm, d).h
    a = h
    flags = []
    for W in [np.asarray(W, np.float64) for W in wq][:-1]:
        z = a @ W.T
        flags.append((np.abs(z) < 2.0 ** -7 * (np.abs(a) @ np.abs(W).T)).ravel())
        a = np.maximum(z, 0.0)
    frac = float(np.mean(np.concatenate(flags)))
    nw = lambda u, v: np.linalg.norm(u - v) / np.linalg.norm(v)
    errs = [nw(dT.cpu().numpy(), rT)]
    gw = dW.cpu().numpy()
    for (off, o, i), rW in zip(sc.weight_slices(), rWs):
        errs.append(nw(gw[off:off + o * i].reshape(o, i), rW))
    print("BF16 shifted backward errors", [round(e, 5) for e in errs], "mask fraction", frac)
    assert errs[-1] <= 1e-2
    assert max(errs[:-1]) <= 3.0 * np.sqrt(frac) + 1e-2
