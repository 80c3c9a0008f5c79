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
