"""The kernels' side of data-parallel training on one GPU: the fused pass of
each rank's shard, normalised by the whole batch's pair count (norm_pairs),
gives the shard's share of the batch loss and gradients, so the shards' sums
equal the full batch's fused pass (what the all-reduce of the ranks forms).
Both precisions; the shards are run one after the other on this GPU."""
import pytest
import torch

from paper_2606_08469_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_08469_gb300 import build
    build.build()


def _rel(a, b):
    return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()


@pytest.mark.parametrize("which,precision,tol", [("train_f32", "f32", 1e-5),
                                                  ("train_bf16", None, 1e-5)])
def test_shard_passes_sum_to_the_batch_pass(which, precision, tol):
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS[which]
    n, world = 3001, 3
    full, _ = WL.train_step_for(cfg, n_pairs=n, precision=precision, fused=True)
    full.fused_pass()
    shards = [WL.data_parallel_train_step(cfg, r, world, n_pairs=n, precision=precision)[0]
              for r in range(world)]
    for s in shards:
        s.fused_pass()
    torch.cuda.synchronize()
    loss = sum(s.loss for s in shards)
    torch.testing.assert_close(loss, full.loss, rtol=1e-6, atol=0)
    gT = sum(s.states[0].grad_t for s in shards)
    gW = sum(s.states[0].grad_w for s in shards)
    assert _rel(gT, full.states[0].grad_t) <= tol
    assert _rel(gW, full.states[0].grad_w) <= tol


def test_data_parallel_step_single_rank_is_the_fused_step():
    """Without a process group DataParallelStep is the fused step itself."""
    from paper_2606_08469_gb300 import dataparallel as D
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_f32"]
    a, _ = WL.train_step_for(cfg, n_pairs=2048, fused=True)
    b, _ = WL.data_parallel_train_step(cfg, 0, 1, n_pairs=2048)
    dp = D.DataParallelStep(b)
    t0 = a.states[0].master_t.clone()
    for _ in range(2):
        a.step()
        dp.step()
    torch.cuda.synchronize()
    torch.testing.assert_close(b.loss, a.loss, rtol=1e-6, atol=0)
    # the updates agree normwise: an Adam update is about lr sign(g), and
    # components whose g lies within the atomics' FP32 rounding of 0 may flip
    ua, ub = a.states[0].master_t - t0, b.states[0].master_t - t0
    assert torch.linalg.norm(ub - ua) <= 1e-3 * torch.linalg.norm(ua)
    with pytest.raises(ValueError):
        D.DataParallelStep(a)                     # no norm_pairs: not a shard step


# ------------------------------------------------- two ranks, one exchange

ROOT = __import__("os").path.dirname(__import__("os").path.dirname(__import__("os").path.abspath(__file__)))
N_DP = 4097


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _dp_rank(rank, world, port, out):
    import os
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_2606_08469_gb300 import api as A
    from paper_2606_08469_gb300 import dataparallel as D
    from paper_2606_08469_gb300 import workloads as WL
    from oracle import octaoctree_oracle as O
    from oracle_helpers import unambiguous_pairs
    from paper_2606_08469_gb300.train import SceneState, TrainStep
    cfg = I.WORKLOADS["train_f32"]
    tree, tables, weights = WL.host_params(cfg)
    ot = O.build_tree(cfg.seed("tree"), cfg.max_depth, cfg.p_base, cfg.R)
    pairs, _ = unambiguous_pairs(ot, tables, weights, I.training_pairs(cfg.seed("queries"), N_DP))
    b, e = D.shard_range(N_DP, rank, world)
    shard = {k: torch.from_numpy(np.ascontiguousarray(getattr(pairs, k)[b:e])).cuda()
             for k in ("x", "omega", "x2", "omega2", "E", "w")}
    st = SceneState(tree, tables, weights, torch.float32, torch.float32, "cuda")
    step = TrainStep([st], [shard], fused=True, norm_pairs=[N_DP])
    dp = D.DataParallelStep(step)
    calls = []
    real = dist.all_reduce
    dist.all_reduce = lambda *a, **k: (calls.append(1), real(*a, **k))[1]
    dp.step()
    dist.all_reduce = real
    torch.cuda.synchronize()
    sc = A.read_scaler(step.scaler)
    st = step.states[0]
    out[rank] = {"loss": float(step.loss.item()), "m_t": st.m_t.cpu().numpy(),
                 "m_w": st.m_w.cpu().numpy(), "master_t": st.master_t.cpu().numpy(),
                 "grad_norm": sc.grad_norm, "skipped": sc.skipped, "collectives": len(calls)}
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_data_parallel_step_matches_oracle_batch():
    """Two processes on this GPU, each with its own shard of a 4,097-pair
    train_f32 batch (gloo all-reduce of CUDA tensors): one DataParallelStep
    (fused pass on the shard, ONE all-reduce of the flat gradient buffer with
    the loss in its tail, Adam).  Pairs with a ReLU mask that binary32 may
    decide either way get a zero residual (oracle_helpers).  Both ranks end
    with identical parameters;
    the batch loss, the gradient read back from Adam's first moment
    (m = (1 - beta1) g after the first step) and the scaler's FP64 gradient
    norm match the FP64 oracle's whole-batch step."""
    import numpy as np
    import torch.multiprocessing as mp
    from oracle import octaoctree_oracle as O
    from paper_2606_08469_gb300 import workloads as WL
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_dp_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    from oracle_helpers import unambiguous_pairs
    cfg = I.WORKLOADS["train_f32"]
    tree, tables, weights = WL.host_params(cfg)
    ot = O.build_tree(cfg.seed("tree"), cfg.max_depth, cfg.p_base, cfg.R)
    pairs, _ = unambiguous_pairs(ot, tables, weights, I.training_pairs(cfg.seed("queries"), N_DP))
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    rgb, _ = O.query_forward(ot, tables, weights, X, Om)
    n = pairs.n
    loss, dLp, dLs = O.residual_loss(rgb[:n], rgb[n:], pairs.E, pairs.w)
    rT, rWs, _ = O.query_backward(ot, tables, weights, X, Om, np.concatenate([dLp, dLs]))
    rW = np.concatenate([w.ravel() for w in rWs])
    b1 = np.float32(1.0) - np.float32(0.9)
    nw = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    for r in range(world):
        g = res[r]
        assert g["collectives"] == 1 and g["skipped"] == 0
        assert abs(g["loss"] - loss) <= 1e-6 * loss, (g["loss"], loss)
        assert nw(g["m_t"] / b1, rT) <= 1e-5 and nw(g["m_w"] / b1, rW) <= 1e-5
        gn = np.sqrt(np.sum(rT ** 2) + np.sum(rW ** 2))
        assert abs(g["grad_norm"] - gn) <= 1e-5 * gn
    np.testing.assert_array_equal(res[0]["master_t"], res[1]["master_t"])
