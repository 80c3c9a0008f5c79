"""A tree larger than every kernel's shared-memory node capacity (a full
octree of 4,681 nodes; the kernels stage at most 2,048): the walk then reads
the node records from global memory.  Same parity bars as the staged path:
node indices and texel addresses bit-exact, FP32 radiance and gradients at
the FP32 bounds, BF16 radiance at 1e-2 normwise."""
import numpy as np
import pytest
import torch

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"
SEED, DEPTH, R, F = 77, 4, [4, 4, 4, 4, 2], 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_08469_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def normwise(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def tree():
    from paper_2606_08469_gb300 import api as A
    t = A.octree_build(SEED, DEPTH, 1.0, R)
    assert t.num_nodes == 1 + 8 + 64 + 512 + 4096 > 2048
    return t, O.build_tree(SEED, DEPTH, 1.0, R)


def _params(t, sigma=0.1):
    tables = I.make_tables(5, t.num_texels, F, sigma)
    weights = I.make_mlp(6, [(DEPTH + 1) * F, 64, 64, 3])
    return tables, weights


def test_fp32_forward_backward_global_walk(tree):
    from paper_2606_08469_gb300 import api as A
    t, ot = tree
    tables, weights = _params(t)
    sc = A.Scene(t, dev(tables), [dev(W) for W in weights], device=DEV)
    x, w = I.uniform_queries(8, 6000)
    rgb, nodes, addr = A.octa_query_fwd(sc, dev(x), dev(w), want_nodes=True, want_addr=True)
    ref, enc = O.query_forward(ot, tables, weights, x, w)
    np.testing.assert_array_equal(nodes.cpu().numpy(), enc.node)
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr)
    assert np.max(np.abs(rgb.cpu().numpy() - ref) / ref) <= 1e-5
    d_rgb = np.random.default_rng(3).normal(size=(len(x), 3)).astype(np.float32)
    dT = torch.zeros(sc.tables.shape, device=DEV)
    dW = torch.zeros(sc.weights.shape, device=DEV)
    A.octa_query_bwd(sc, dev(x), dev(w), dev(d_rgb), [(dT, dW)])
    rT, rWs, _ = O.query_backward(ot, tables, weights, x, w, d_rgb)
    assert normwise(dT.cpu().numpy(), rT) <= 1e-5
    gw = dW.cpu().numpy()
    for (off, o, i), rW in zip(sc.weight_slices(), rWs):
        assert normwise(gw[off:off + o * i].reshape(o, i), rW) <= 1e-5


def test_fp32_fused_training_pass_global_walk(tree):
    """The fused FP32 training pass against forward + residual_loss +
    backward, both walking in global memory."""
    from paper_2606_08469_gb300 import train as TR
    t, ot = tree
    tables, weights = _params(t, sigma=0.01)
    pairs = I.training_pairs(9, 3001)
    steps = []
    for fused in (False, True):
        st = TR.SceneState(t, tables, weights, torch.float32, torch.float32, DEV)
        p = {k: dev(getattr(pairs, k)) for k in ("x", "omega", "x2", "omega2", "E", "w")}
        steps.append(TR.TrainStep([st], [p], fused=fused))
    a, b = steps
    a.forward()
    a.loss_and_grad()
    a.backward()
    b.fused_pass()
    torch.cuda.synchronize()
    torch.testing.assert_close(b.loss, a.loss, rtol=1e-6, atol=0)
    for ga, gb in ((a.states[0].grad_t, b.states[0].grad_t), (a.states[0].grad_w, b.states[0].grad_w)):
        assert (torch.linalg.norm(gb - ga) / torch.linalg.norm(ga)).item() <= 1e-5


def test_bf16_forward_and_encode_global_walk(tree):
    from paper_2606_08469_gb300 import api as A
    t, ot = tree
    tables, weights = _params(t)
    sc = A.Scene(t, dev(tables).half(), [dev(W).to(torch.bfloat16) for W in weights], device=DEV)
    x, w = I.uniform_queries(10, 5000)
    rgb, nodes, addr = A.octa_query_fwd(sc, dev(x), dev(w), want_nodes=True, want_addr=True)
    ref, enc = O.query_forward(ot, tables, weights, x, w)
    np.testing.assert_array_equal(nodes.cpu().numpy(), enc.node)
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr)
    assert normwise(rgb.cpu().numpy(), ref) <= 1e-2
    tq = tables.astype(np.float16).astype(np.float32)
    feat, fn, fa = A.octa_encode(sc, dev(x), dev(w), want_nodes=True, want_addr=True)
    np.testing.assert_array_equal(fn.cpu().numpy(), enc.node)
    np.testing.assert_array_equal(fa.cpu().numpy(), enc.addr)
    ref_h = O.encode_features(ot, tq, x, w).h
    bound = 4 * 2.0 ** -24 * max(R) * np.abs(tq).max()
    np.testing.assert_allclose(feat.cpu().numpy(), ref_h, rtol=0, atol=bound + 1e-7)
