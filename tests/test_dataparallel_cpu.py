"""Data-parallel training logic on CPU ranks (gloo, two ranks): each rank
takes its shard of the batch, forms its share of the batch's loss gradient
(normalised by the whole batch's pair count) and back-propagates it with the
FP64 oracle; the ranks' all-reduced sums must equal the oracle's gradients of
the whole batch.  The GPU side of the same normalisation (norm_pairs in the
fused pass) is checked in test_gpu_dataparallel.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_PAIRS = 301


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from oracle import octaoctree_oracle as O
    from paper_2606_08469_gb300 import inputs as I
    cfg = I.WORKLOADS["forward_small"]
    ot = O.build_tree(cfg.seed("tree"), cfg.max_depth, cfg.p_base, cfg.R)
    tables = I.make_tables(cfg.seed("tables"), ot.num_texels, cfg.F, 0.3)
    weights = I.make_mlp(cfg.seed("mlp"), [ot.num_levels * cfg.F, 32, 32, 3])
    pairs = I.training_pairs(77, N_PAIRS)
    return O, ot, tables, weights, pairs


def _grads(O, ot, tables, weights, pairs, b, e, n_norm):
    """Gradient of (1 / (3 n_norm)) * sum over pairs [b, e) of r^2."""
    sl = slice(b, e)
    Lp, _ = O.query_forward(ot, tables, weights, pairs.x[sl], pairs.omega[sl])
    Ls, _ = O.query_forward(ot, tables, weights, pairs.x2[sl], -pairs.omega2[sl])
    loss, dp, ds = O.residual_loss(Lp, Ls, pairs.E[sl], pairs.w[sl])
    f = (e - b) / n_norm                       # own-count mean -> share of the batch
    gTp, gWp, _ = O.query_backward(ot, tables, weights, pairs.x[sl], pairs.omega[sl], dp * f)
    gTs, gWs, _ = O.query_backward(ot, tables, weights, pairs.x2[sl], -pairs.omega2[sl], ds * f)
    return loss * f, gTp + gTs, [a + c for a, c in zip(gWp, gWs)]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2606_08469_gb300 import dataparallel as D
    O, ot, tables, weights, pairs = _problem()
    b, e = D.shard_range(N_PAIRS, rank, world)
    loss, gT, gWs = _grads(O, ot, tables, weights, pairs, b, e, N_PAIRS)
    ts = [torch.tensor([loss], dtype=torch.float64), torch.from_numpy(gT)] + \
        [torch.from_numpy(g) for g in gWs]
    D.allreduce_sum(ts)
    out[rank] = [t.numpy().copy() for t in ts]
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_gradients_sum_to_the_batch_gradient():
    import sys
    sys.path.insert(0, ROOT)
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    O, ot, tables, weights, pairs = _problem()
    loss, gT, gWs = _grads(O, ot, tables, weights, pairs, 0, N_PAIRS, N_PAIRS)
    for r in range(world):
        got = res[r]
        assert abs(got[0][0] - loss) <= 1e-12 * loss
        np.testing.assert_allclose(got[1], gT, rtol=0, atol=1e-12 * np.abs(gT).max())
        for g, ref in zip(got[2:], gWs):
            np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_shard_ranges_partition_the_batch():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2606_08469_gb300 import dataparallel as D
    for n in (0, 1, 7, 301, 1 << 20):
        for world in (1, 2, 3, 8):
            spans = [D.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.shard_range(5, 2, 2)


def _flat_rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2606_08469_gb300 import dataparallel as D
    g = np.random.default_rng(100 + rank)
    flat = torch.from_numpy(g.normal(size=1000).astype(np.float32))
    flat[-4:] = 0.0                                    # the two losses' slots
    losses = torch.tensor([0.123456789012345 * (rank + 1), 1e-3 / (rank + 3)], dtype=torch.float64)
    calls = []
    real = dist.all_reduce
    dist.all_reduce = lambda *a, **k: (calls.append(1), real(*a, **k))[1]
    D.allreduce_flat(flat, losses)
    dist.all_reduce = real
    out[rank] = (flat.numpy().copy(), losses.numpy().copy(), len(calls))
    dist.barrier()
    dist.destroy_process_group()


def test_flat_exchange_one_collective_two_ranks():
    """A data-parallel step's exchange: the gradients and the FP64 losses
    (as FP32 hi/lo pairs in the buffer's tail) in ONE all-reduce; the sum
    of the ranks' losses comes back to about binary32 rounding of the sum."""
    import sys
    sys.path.insert(0, ROOT)
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_flat_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    want = sum(np.random.default_rng(100 + r).normal(size=1000).astype(np.float32) for r in range(world))
    want_loss = np.array([0.123456789012345 * 3, 1e-3 / 3 + 1e-3 / 4])
    for r in range(world):
        flat, losses, calls = res[r]
        assert calls == 1
        np.testing.assert_allclose(flat[:-4], want[:-4], rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(losses, want_loss, rtol=1e-7, atol=0)
