"""The full query form on the GPU (octa_encode with OCTA_FORM_TRILINEAR_VERTEX:
Eq. 10 eight-cell renormalised trilinear blend with Eq. 6 barycentric
interpolation on vertex maps) against the FP64 oracle: the 24 vertex entries
per level bit-exact, features within the binary32 bound of a 24-term blend."""
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
        A.octa_query_fwd(sc, dev(x), dev(w))             # the decoder path takes the cell form only
    with pytest.raises(L.OctaError):
        A.octa_encode(sc, dev(x), dev(w), want_nodes=True)
