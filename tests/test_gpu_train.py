"""GPU parity of the training-side entry points (residual_loss, adam_step,
dynamic loss scaling) and of a whole FP32 training step, against the oracle."""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_08469_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("rhs_grad,n", [(True, 1), (True, 100003), (False, 4096)])
def test_residual_loss_matches_oracle(rhs_grad, n):
    from paper_2606_08469_gb300 import api as A
    from paper_2606_08469_gb300 import _lib as L
    g = np.random.default_rng(n)
    Lp, Ls = (g.uniform(0.2, 3.0, size=(n, 3)).astype(np.float32) for _ in range(2))
    E = (g.random((n, 3)) * (g.random((n, 1)) < 0.05)).astype(np.float32)
    w = g.random((n, 3)).astype(np.float32)
    scaler = A.make_scaler(2.0 ** 15, 2000)
    dLp = torch.empty((n, 3), device=DEV)
    dLs = torch.full((n, 3), 7.0, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    ws = A.workspace(L.OCTA_OP_LOSS, n)
    for _ in range(2):                         # the workspace is reusable
        A.residual_loss(dev(Lp), dev(Ls), dev(E), dev(w), dLp, dLs, loss, ws, 1e-2, rhs_grad, scaler)
    rl, rdp, rds = O.residual_loss(Lp, Ls, E, w, 1e-2, rhs_grad, 2.0 ** 15)
    assert abs(loss.item() - rl) <= 1e-6 * rl
    np.testing.assert_allclose(dLp.cpu().numpy(), rdp, rtol=2e-5, atol=1e-7 * np.abs(rdp).max())
    np.testing.assert_allclose(dLs.cpu().numpy(), rds, rtol=2e-5, atol=1e-7 * np.abs(rdp).max())


def test_adam_matches_oracle_and_scaler():
    from paper_2606_08469_gb300 import api as A
    from paper_2606_08469_gb300 import _lib as L
    g = np.random.default_rng(0)
    n1, n2 = 1000, 37
    p1 = g.normal(size=n1).astype(np.float32)
    p2 = g.normal(size=n2).astype(np.float32)
    P1, P2 = dev(p1), dev(p2)
    G1, G2 = torch.zeros(n1, device=DEV), torch.zeros(n2, device=DEV)
    M1, V1, M2, V2 = (torch.zeros(n, device=DEV) for n in (n1, n1, n2, n2))
    W1 = torch.zeros(n1, dtype=torch.float16, device=DEV)
    W2 = torch.zeros(n2, dtype=torch.bfloat16, device=DEV)
    groups = [A.ParamGroup(P1, G1, M1, V1, 1e-2, W1), A.ParamGroup(P2, G2, M2, V2, 1e-3, W2)]
    S = 2.0 ** 15
    scaler = A.make_scaler(S, growth_interval=2)
    ws = A.workspace(L.OCTA_OP_ADAM, n1 + n2)
    r1, r2 = p1.astype(np.float64), p2.astype(np.float64)
    m1 = v1 = np.zeros(n1)
    m2 = v2 = np.zeros(n2)
    t = 0
    scales = [S]
    for step in range(5):
        g1 = g.normal(size=n1).astype(np.float32)
        g2 = g.normal(size=n2).astype(np.float32)
        inject = step == 2
        if inject:
            g2[5] = np.inf                     # host-injected overflow
        G1.copy_(dev(g1 * np.float32(scales[-1])))
        G2.copy_(dev(g2 * np.float32(scales[-1])))
        A.adam_step(groups, scaler, ws)
        st = A.read_scaler(scaler)
        assert st.skipped == int(inject)
        assert torch.count_nonzero(G1).item() == 0 and torch.count_nonzero(G2).item() == 0
        if not inject:
            t += 1
            r1, m1, v1 = O.adam_update(r1, g1, m1, v1, t, 1e-2)
            r2, m2, v2 = O.adam_update(r2, g2, m2, v2, t, 1e-3)
            assert abs(st.grad_norm - np.sqrt(np.sum(g1.astype(np.float64) ** 2) +
                                              np.sum(g2.astype(np.float64) ** 2))) < 1e-5 * st.grad_norm
        assert st.step == t
        scales.append(st.scale)
        np.testing.assert_allclose(P1.cpu().numpy(), r1, rtol=0, atol=2e-6)
        np.testing.assert_allclose(P2.cpu().numpy(), r2, rtol=0, atol=2e-6)
        np.testing.assert_array_equal(W1.cpu().numpy(), P1.cpu().numpy().astype(np.float16))
    # trajectory: finite, finite -> grow, overflow -> halve, finite, finite -> grow
    ref = O.LossScaler(S, growth_interval=2)
    want = [S]
    for step in range(5):
        ref.update(step != 2)
        want.append(ref.scale)
    assert scales == want


def _oracle_state(tables, weights):
    T = tables.astype(np.float64)
    Ws = [W.astype(np.float64) for W in weights]
    return O.TrainState(T, Ws, np.zeros_like(T), np.zeros_like(T), [np.zeros_like(w) for w in Ws],
                        [np.zeros_like(w) for w in Ws])


def _update_err(new_gpu, new_ref, old):
    """Normwise error of the parameter update.  Elementwise comparison is
    ill-conditioned: Adam's first steps move every parameter by about
    lr * sign(g), so a gradient component within its FP32 error of zero can
    flip; the update as a whole is what the gradients determine."""
    d_ref = new_ref - old
    return np.linalg.norm((new_gpu - old) - d_ref) / np.linalg.norm(d_ref)


@pytest.mark.parametrize("fused", [False, True])
def test_train_step_matches_oracle(fused):
    """Two full FP32 steps (fwd, loss, bwd, Adam + scaler) of config-1 shapes
    on 4096 pairs vs the oracle's step; fused = the one-launch training pass
    of the FP32 engine in place of forward + residual_loss + backward."""
    from paper_2606_08469_gb300 import api as A
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_f32"]
    step, (tree, tables, weights, pairs) = WL.train_step_for(cfg, n_pairs=4096, fused=fused)
    ot = O.build_tree(cfg.seed("tree"), cfg.max_depth, cfg.p_base, cfg.R)
    st = _oracle_state(tables, weights)
    scaler = O.LossScaler()
    for _ in range(2):
        old_t = st.tables.copy()
        old_w = np.concatenate([w.reshape(-1) for w in st.weights])
        step.step()
        torch.cuda.synchronize()
        loss, gn, skipped = O.train_step(ot, st, pairs, scaler)
        sc = A.read_scaler(step.scaler)
        assert not skipped and sc.skipped == 0
        assert abs(step.loss.item() - loss) <= 1e-5 * loss
        assert abs(sc.grad_norm - gn) <= 1e-5 * gn
        gt = step.states[0].master_t.cpu().numpy()
        gw = step.states[0].master_w.cpu().numpy()
        W = np.concatenate([w.reshape(-1) for w in st.weights])
        assert _update_err(gt, st.tables, old_t) <= 1e-3
        assert _update_err(gw, W, old_w) <= 1e-3
        # the same start point for the next step on both sides
        st.tables = gt.astype(np.float64)
        off = 0
        for i, w in enumerate(st.weights):
            st.weights[i] = gw[off:off + w.size].reshape(w.shape).astype(np.float64)
            off += w.size


def test_train_step_full_config1_loss_and_samples():
    """The full 262,144-pair config-1 step on the GPU: the forward on sampled
    queries and the loss value of the whole batch vs the oracle."""
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_f32"]
    step, (tree, tables, weights, pairs) = WL.train_step_for(cfg)
    step.forward()
    step.loss_and_grad()
    torch.cuda.synchronize()
    ot = O.build_tree(cfg.seed("tree"), cfg.max_depth, cfg.p_base, cfg.R)
    N = pairs.n
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    rgb = step.rgb.cpu().numpy()
    idx = np.random.default_rng(0).choice(2 * N, 4096, replace=False)
    ref, _ = O.query_forward(ot, tables, weights, X[idx], Om[idx])
    assert np.max(np.abs(rgb[idx] - ref) / ref) <= 1e-5
    ref_all, _ = O.query_forward(ot, tables, weights, X, Om)
    loss, _, _ = O.residual_loss(ref_all[:N], ref_all[N:], pairs.E, pairs.w)
    assert abs(step.loss.item() - loss) <= 1e-5 * loss
    step.backward()
    step.optimizer()
    torch.cuda.synchronize()
    assert torch.isfinite(step.states[0].master_t).all()


def test_train_step_graph_replay_equals_eager():
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_f32"]
    a, host = WL.train_step_for(cfg, n_pairs=8192)
    b, _ = WL.train_step_for(cfg, n_pairs=8192)
    t0 = torch.from_numpy(host[1]).to(DEV)
    a.step()                                   # eager warm-up of every kernel
    b.step()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            b.step()
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        a.step()
        graph.replay()
    torch.cuda.synchronize()
    # atomics make the summation order (not the sum) differ between runs
    torch.testing.assert_close(a.loss, b.loss, rtol=1e-5, atol=0)
    ta, tb = a.states[0].master_t, b.states[0].master_t
    assert torch.linalg.norm(ta - tb) <= 1e-3 * torch.linalg.norm(ta - t0)


def _grad_err(a, b):
    """Largest normwise difference of the table and weight gradients."""
    e = 0.0
    for sa, sb in zip(a.states, b.states):
        for ga, gb in ((sa.grad_t, sb.grad_t), (sa.grad_w, sb.grad_w)):
            e = max(e, (torch.linalg.norm(ga - gb) / torch.linalg.norm(gb)).item())
    return e


@pytest.mark.parametrize("rhs_grad", [True, False])
def test_fused_f32_pass_matches_unfused(rhs_grad):
    """The FP32 engine's fused training pass (64-pair tiles, in-tile Eq. 14
    gradient) against octa_query_fwd + residual_loss + octa_query_bwd on a
    ragged batch (4097 pairs: a one-pair tail tile).  Both run the same FP32
    arithmetic; only the atomics' summation order differs."""
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_f32"]
    a, _ = WL.train_step_for(cfg, n_pairs=4097, rhs_grad=rhs_grad)
    b, _ = WL.train_step_for(cfg, n_pairs=4097, rhs_grad=rhs_grad, fused=True)
    a.forward()
    a.loss_and_grad()
    a.backward()
    b.fused_pass()
    torch.cuda.synchronize()
    torch.testing.assert_close(b.loss, a.loss, rtol=1e-6, atol=0)
    err = _grad_err(b, a)
    print("fused vs unfused FP32 gradients", err)
    assert err <= 1e-5


def test_fused_f32_pass_batched_scenes():
    """Eight scenes of uneven size (FP32 copies of the batched workload's
    parameters) in one fused FP32 launch vs the unfused path, per scene."""
    from paper_2606_08469_gb300 import workloads as WL
    counts = [3000, 1, 64, 65, 700, 129, 5, 2048]
    a, _ = WL.batched_train_step(counts=counts, precision="f32")
    b, _ = WL.batched_train_step(counts=counts, precision="f32", fused=True)
    a.forward()
    a.loss_and_grad()
    a.backward()
    b.fused_pass()
    torch.cuda.synchronize()
    la, lb = a.loss.cpu().numpy(), b.loss.cpu().numpy()
    np.testing.assert_allclose(lb, la, rtol=1e-6, atol=0)
    for sa, sb in zip(a.states, b.states):
        for ga, gb in ((sa.grad_t, sb.grad_t), (sa.grad_w, sb.grad_w)):
            assert (torch.linalg.norm(gb - ga) / torch.linalg.norm(ga)).item() <= 1e-5


def test_pair_inputs_can_be_swapped():
    """A fused step reading a copy of its pair arrays (set_pair_inputs, as the
    double-buffered end-to-end loop does) gives the same loss and gradients;
    arrays of another shape are refused."""
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_f32"]
    a, _ = WL.train_step_for(cfg, n_pairs=1000, fused=True)
    b, _ = WL.train_step_for(cfg, n_pairs=1000, fused=True)
    copies = {k: t.clone() for k, t in b.pair_inputs().items()}
    b.set_pair_inputs(copies)
    a.fused_pass()
    b.fused_pass()
    torch.cuda.synchronize()
    torch.testing.assert_close(b.loss, a.loss, rtol=1e-6, atol=0)
    assert torch.linalg.norm(b.states[0].grad_t - a.states[0].grad_t) <= \
        1e-5 * torch.linalg.norm(a.states[0].grad_t)
    bad = dict(copies, Px=copies["Px"][:-1])
    with pytest.raises(ValueError):
        b.set_pair_inputs(bad)


def test_measure_mma_reports_cycles():
    """The MMA microbenchmark completes and reports positive cycle counts,
    the completion after the issue, more cycles for wider N."""
    import torch
    from paper_2606_08469_gb300 import api
    lib = api._lib()
    out = torch.zeros(3, dtype=torch.int64, device="cuda")
    got = {}
    for n in (64, 256):
        api.L.check(lib.octa_measure_mma(api._ptr(out), n, 4, 11, 1, api._stream()),
                    "octa_measure_mma")
        issue, done, ok = out.tolist()
        assert ok == 1 and 0 < issue <= done
        got[n] = done
    assert got[256] > got[64]
    api.L.check(lib.octa_measure_mma(api._ptr(out), 64, 5, 3, 2, api._stream()), "octa_measure_mma")
    assert out.tolist()[2] == 1
