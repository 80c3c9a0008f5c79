"""GPU parity of the BF16 tensor-core path against the FP64 oracle.

Binding bound: radiance within 1e-2 normwise of the FP64 oracle evaluated
with the FP32 master parameters (tables and weights before quantisation).
Node indices and texel addresses stay bit-exact (the address path is the
same canonical binary32 sequence).  The error against FP64 on the quantised
parameters (FP16 tables and BF16 weights widened exactly) isolates the
arithmetic: BF16 operands with FP32 accumulation, bounded here by 6e-3."""
import numpy as np
import pytest
import torch

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL_E2E = 1e-2
TOL_ARITH = 6e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_08469_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def normwise(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_bf16_scene(seed, depth, R, F, sigma, hidden, wscale=1.0, tseed=2000, wseed=3000,
                    tdt=torch.float16):
    from paper_2606_08469_gb300 import api as A
    tree = A.octree_build(seed, depth, 0.6, R)
    tables = I.make_tables(tseed, tree.num_texels, F, sigma)
    weights = [W * np.float32(wscale) for W in I.make_mlp(wseed, [(depth + 1) * F] + hidden + [3])]
    sc = A.Scene(tree, dev(tables).to(tdt).contiguous(),
                 [dev(W).to(torch.bfloat16) for W in weights], device=DEV)
    tq = tables.astype(np.float16).astype(np.float32) if tdt == torch.float16 else tables
    wq = [bf16_round(W) for W in weights]
    return sc, O.build_tree(seed, depth, 0.6, R), tables, weights, tq, wq


def check_forward(sc, ot, tables, weights, tq, wq, x, w, counts=None, tol_arith=TOL_ARITH):
    from paper_2606_08469_gb300 import api as A
    rgb, nodes, addr = A.octa_query_fwd(sc, dev(x), dev(w), counts, want_nodes=True, want_addr=True)
    rgb = rgb.cpu().numpy()
    ref, enc = O.query_forward(ot, tables, weights, x, w)
    refq, _ = O.query_forward(ot, tq, wq, x, w)
    np.testing.assert_array_equal(nodes.cpu().numpy(), enc.node)
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr)
    e2e, arith = normwise(rgb, ref), normwise(rgb, refq)
    assert e2e <= TOL_E2E, e2e
    assert arith <= tol_arith, arith
    return e2e, arith


def test_bf16_forward_config3_gbuffer_sample():
    """Config [3]: 1280x720 G-buffer queries, depth-8 tree, FP16 features,
    decoder 72-64-64-3 in BF16; all queries on the GPU, a 65,536-query
    sample (every 14th pixel) against the oracle."""
    from paper_2606_08469_gb300 import api as A
    cfg = I.CONFIGS[3]
    sc, ot, tables, weights, tq, wq = make_bf16_scene(cfg.seed("tree"), 8, cfg.R, 8, cfg.sigma,
                                                      [64, 64], tseed=cfg.seed("tables"),
                                                      wseed=cfg.seed("mlp"))
    x, w = I.gbuffer_queries(cfg.seed("queries"), 1280, 720)
    rgb, _, _ = A.octa_query_fwd(sc, dev(x), dev(w))
    idx = np.arange(0, len(x), 14)[:65536]
    ref, _ = O.query_forward(ot, tables, weights, x[idx], w[idx])
    assert normwise(rgb.cpu().numpy()[idx], ref) <= TOL_E2E
    check_forward(sc, ot, tables, weights, tq, wq, x[idx[:8192]], w[idx[:8192]])


@pytest.mark.parametrize("shape", ["cfg0", "cfg1", "cfg2"])
@pytest.mark.parametrize("n", [1, 129, 5000])
def test_bf16_forward_shapes(shape, n):
    """Every built decoder shape, features drawn wide (sigma 0.3, weights x2)
    so that the decoder is far from linear, ragged batch sizes."""
    if shape == "cfg0":
        cfg, hidden, F = I.CONFIGS[0], [32, 32], 4
    elif shape == "cfg1":
        cfg, hidden, F = I.CONFIGS[1], [64, 64], 8
    else:
        cfg, hidden, F = I.CONFIGS[2], [64, 64, 64], 8
    sc, ot, tables, weights, tq, wq = make_bf16_scene(cfg.seed("tree"), cfg.max_depth, cfg.R, F,
                                                      0.3, hidden, wscale=2.0)
    x, w = I.uniform_queries(500 + n, n)
    check_forward(sc, ot, tables, weights, tq, wq, x, w)


def test_bf16_forward_fp32_tables():
    cfg = I.CONFIGS[1]
    sc, ot, tables, weights, tq, wq = make_bf16_scene(cfg.seed("tree"), cfg.max_depth, cfg.R, 8,
                                                      0.3, [64, 64], wscale=2.0, tdt=torch.float32)
    x, w = I.uniform_queries(61, 3000)
    check_forward(sc, ot, tables, weights, tq, wq, x, w)


def test_bf16_forward_batched_scenes():
    """Scenes of depth 4, 6 and 9 (K*F = 40, 56, 80 padded to 80) in one
    launch, each with its own BF16 decoder."""
    from paper_2606_08469_gb300 import api as A
    specs = [(1400, 4), (1402, 6), (1407, 9)]
    counts = [700, 4000, 1301]
    parts = []
    for s, ((seed, depth), n) in enumerate(zip(specs, counts)):
        parts.append(make_bf16_scene(seed, depth, I.R_DEEP[:depth + 1], 8, 0.3, [64, 64],
                                     wscale=2.0, tseed=2400 + s, wseed=3400 + s))
    xs, ws = zip(*[I.uniform_queries(4400 + s, n) for s, n in enumerate(counts)])
    X, W = np.concatenate(xs), np.concatenate(ws)
    rgb, nodes, addr = A.octa_query_fwd([p[0] for p in parts], dev(X), dev(W), counts,
                                        want_nodes=True, want_addr=True)
    rgb, nodes, addr = rgb.cpu().numpy(), nodes.cpu().numpy(), addr.cpu().numpy()
    off = 0
    for s, n in enumerate(counts):
        sc, ot, tables, weights, tq, wq = parts[s]
        sl = slice(off, off + n)
        ref, enc = O.query_forward(ot, tables, weights, xs[s], ws[s])
        K = ot.num_levels
        np.testing.assert_array_equal(nodes[sl, :K], enc.node)
        np.testing.assert_array_equal(addr[sl, :K], enc.addr)
        assert normwise(rgb[sl], ref) <= TOL_E2E
        off += n
