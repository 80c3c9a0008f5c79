"""Launch knobs change how work is spread, never the results; the autotuner
picks a setting and caches it."""
import json

import numpy as np
import pytest
import torch

from paper_2606_08469_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _reset():
    from paper_2606_08469_gb300 import build
    build.build()
    from paper_2606_08469_gb300 import autotune as T
    T.set_tuning(None)
    yield
    T.set_tuning(None)


def test_forward_results_independent_of_knobs():
    from paper_2606_08469_gb300 import api as A
    from paper_2606_08469_gb300 import autotune as T
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["gbuffer_frame"]
    sc, _ = WL.forward_scene(cfg)
    x, w = I.uniform_queries(3, 50000)
    X, W = WL.to_dev(x), WL.to_dev(w)
    ref, rn, ra = A.octa_query_fwd(sc, X, W, want_nodes=True, want_addr=True)
    counts = [777, len(x) - 777]              # two scenes, a ragged first tile
    ref2, _, _ = A.octa_query_fwd([sc, sc], X, W, counts)
    for setting in ({"fwd_ctas_per_sm": 1}, {"fwd_ctas_per_sm": 2, "fwd_order": 1},
                    {"fwd_order": 1}, {"fwd_threads_per_query": 2},
                    {"fwd_threads_per_query": 2, "fwd_order": 1, "fwd_ctas_per_sm": 3},
                    {"fwd_run": 3}, {"fwd_run": 8, "fwd_ctas_per_sm": 2},
                    {"fwd_run": 64, "fwd_threads_per_query": 2}, {"l1_carveout": 2},
                    {"l1_carveout": 2, "fwd_threads_per_query": 2}, {"l1_carveout": 1},
                    {"fwd_threads_per_query": 1}, {"fwd_threads_per_query": 1, "fwd_run": 4}):
        T.set_tuning(setting)
        got, gn, ga = A.octa_query_fwd(sc, X, W, want_nodes=True, want_addr=True)
        torch.testing.assert_close(got, ref, rtol=0, atol=0)
        assert torch.equal(gn, rn) and torch.equal(ga, ra)
        got2, _, _ = A.octa_query_fwd([sc, sc], X, W, counts)
        torch.testing.assert_close(got2, ref2, rtol=0, atol=0)


def test_training_results_independent_of_order():
    from paper_2606_08469_gb300 import autotune as T
    from paper_2606_08469_gb300 import workloads as WL
    counts = [3000, 129, 20000, 64, 64, 64, 64, 64]
    a, _ = WL.batched_train_step(counts=counts, fused=True)
    b, _ = WL.batched_train_step(counts=counts, fused=True)
    a.fused_pass()
    torch.cuda.synchronize()
    for setting in ({"train_order": 1}, {"train_run": 3}, {"train_run": 16, "train_order": 2}):
        for st in b.states:
            st.grad_t.zero_()
            st.grad_w.zero_()
        T.set_tuning(setting)
        b.fused_pass()
        torch.cuda.synchronize()
        torch.testing.assert_close(b.loss, a.loss, rtol=1e-6, atol=0)
        for sa, sb in zip(a.states, b.states):
            assert torch.linalg.norm(sa.grad_t - sb.grad_t) <= 1e-5 * torch.linalg.norm(sa.grad_t)
            assert torch.linalg.norm(sa.grad_w - sb.grad_w) <= 1e-5 * torch.linalg.norm(sa.grad_w)


def test_autotune_picks_and_caches(tmp_path):
    from paper_2606_08469_gb300 import api as A
    from paper_2606_08469_gb300 import autotune as T
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["gbuffer_frame"]
    sc, _ = WL.forward_scene(cfg)
    x, w = I.uniform_queries(4, 100000)
    X, W = WL.to_dev(x), WL.to_dev(w)
    rgb = torch.empty((len(x), 3), device="cuda")
    fn = lambda: A.octa_query_fwd(sc, X, W, rgb=rgb)
    cache = str(tmp_path / "tune.json")
    best, rep = T.autotune(fn, {"fwd_ctas_per_sm": [2, 4], "fwd_order": [1, 2]}, "test-fwd", cache,
                           reps=3)
    assert len(rep["trials"]) == 4 and rep["best_ms"] == min(t["ms"] for t in rep["trials"])
    assert T.get_tuning()["fwd_ctas_per_sm"] == best["fwd_ctas_per_sm"]
    with open(cache) as f:
        assert any(k.endswith("|test-fwd") for k in json.load(f))
    best2, rep2 = T.autotune(fn, {"fwd_ctas_per_sm": [2, 4]}, "test-fwd", cache)
    assert best2 == best and rep2["best_ms"] == rep["best_ms"]     # served from the cache


@pytest.mark.parametrize("name,dtypes", [("gbuffer_frame", (torch.bfloat16, torch.float32)),
                                         ("forward_small", (torch.float32,))])
def test_encode_results_independent_of_gather_stages(name, dtypes):
    """The texel ring (gather_stages 2..4, cp.async into shared memory) gives
    the register window's features, node indices and texel addresses bit for
    bit: FP16 texels of 8 features and FP32 texels of 4 (both 16 bytes)."""
    from paper_2606_08469_gb300 import api as A
    from paper_2606_08469_gb300 import autotune as T
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS[name]
    sc, _ = WL.forward_scene(cfg)
    x, w = I.uniform_queries(5, 40000)
    X, W = WL.to_dev(x), WL.to_dev(w)
    counts = [333, len(x) - 333]              # two scenes, a ragged first tile
    for dt in dtypes:
        T.set_tuning({"gather_stages": 1})
        ref, rn, ra = A.octa_encode(sc, X, W, feat_dtype=dt, want_nodes=True, want_addr=True)
        ref2, _, _ = A.octa_encode([sc, sc], X, W, counts, feat_dtype=dt)
        for setting in ({"gather_stages": 2}, {"gather_stages": 3},
                        {"gather_stages": 4, "encode_ctas_per_sm": 2},
                        {"gather_stages": 3, "fwd_order": 1, "fwd_run": 4},
                        {"l1_carveout": 1}, {"l1_carveout": 2, "gather_stages": 2},
                        {"l1_carveout": 1, "gather_stages": 4, "fwd_run": 3}):
            T.set_tuning(setting)
            got, gn, ga = A.octa_encode(sc, X, W, feat_dtype=dt, want_nodes=True, want_addr=True)
            assert torch.equal(got, ref), setting
            assert torch.equal(gn, rn) and torch.equal(ga, ra)
            got2, _, _ = A.octa_encode([sc, sc], X, W, counts, feat_dtype=dt)
            assert torch.equal(got2, ref2), setting


def test_encode_mixed_row_layouts_in_one_call():
    """Scenes of 5 and 7 levels in one call with the deeper scene's row
    stride: its tiles leave through per-warp bulk copies, the shallower
    scene's (rows shorter than the stride) through the strided copy, and a
    persistent CTA alternates between the two; the features equal each
    scene encoded alone, bit for bit, whatever the work order."""
    from paper_2606_08469_gb300 import api as A
    from paper_2606_08469_gb300 import autotune as T
    scenes = []
    for s, depth in enumerate((4, 6)):
        R = I.R_DEEP[:depth + 1]
        tree = A.octree_build(1400 + 2 * s, depth, 0.6, R)
        tables = I.make_tables(2400 + s, tree.num_texels, 8, 0.3)
        weights = I.make_mlp(3400 + s, [(depth + 1) * 8, 64, 64, 3])
        scenes.append(A.Scene(tree, torch.from_numpy(tables).cuda(),
                              [torch.from_numpy(W).cuda() for W in weights], device="cuda"))
    counts = [40000, 50000]
    xs, ws = zip(*[I.uniform_queries(90 + s, n) for s, n in enumerate(counts)])
    X = torch.from_numpy(np.concatenate(xs)).cuda()
    Wd = torch.from_numpy(np.concatenate(ws)).cuda()
    for dt in (torch.bfloat16, torch.float32):
        T.set_tuning(None)
        alone = [A.octa_encode(scenes[s], torch.from_numpy(xs[s]).cuda(),
                               torch.from_numpy(ws[s]).cuda(), feat_dtype=dt)[0]
                 for s in range(2)]
        for setting in (None, {"encode_ctas_per_sm": 1}, {"encode_ctas_per_sm": 1, "fwd_order": 1},
                        {"encode_ctas_per_sm": 2, "fwd_run": 3}):
            T.set_tuning(setting)
            feat, _, _ = A.octa_encode(scenes, X, Wd, counts, feat_dtype=dt)
            assert torch.equal(feat[:counts[0], :40], alone[0]), setting
            assert not feat[:counts[0], 40:].any()
            assert torch.equal(feat[counts[0]:], alone[1]), setting
