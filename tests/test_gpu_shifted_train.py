"""Training the paper's full model on the GPU: the disparity-shifted lookup's
backward with dL/dd (FP32 engine and tcgen05 kernels), g_psi's backward
(octa_disparity_bwd) and a whole shifted-form training step (predictor,
shifted lookup, decoder, Eq. 14, every gradient) against the FP64 oracle.

Integers that floating point decides are compared where both sides decide
them alike: the decoder's and g_psi's ReLU masks (queries with a hidden
pre-activation within 2^-16 sum|w||a| of zero carry no gradient) and, in the
whole step, the shifted lookup's triangles (the GPU's disparity comes from
its own FP32 g_psi, the oracle's from FP64 rounded to binary32, so pairs
whose decisions change when d moves by 2^-16 relative carry no gradient).
The sets are found by the oracle alone (tests/oracle_helpers.py)."""
import numpy as np
import pytest
import torch

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I
from oracle_helpers import (decoder_ambiguous, lookup_unstable, neutralise_pairs,
                            predictor_ambiguous)

pytestmark = pytest.mark.gpu
DEV = "cuda"
SMS = 152
F32 = np.float32


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_08469_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def normwise(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def weight_errors(gW, rWs):
    out, off = [], 0
    for rW in rWs:
        out.append(normwise(gW[off:off + rW.size].reshape(rW.shape), rW))
        off += rW.size
    return out


def _tree(seed, depth, V):
    from paper_2606_08469_gb300 import api as A
    return A.octree_build(seed, depth, 0.6, V), O.build_tree(seed, depth, 0.6, V)


def _queries(seed, n, dmax=6.0):
    g = I.rng(seed)
    x = g.random((n, 3)).astype(F32)
    w = I.unit_vectors(g, n).astype(F32)
    nrm = (I.unit_vectors(g, n) * g.uniform(0.5, 2.0, (n, 1))).astype(F32)
    d = g.uniform(0.0, dmax, n).astype(F32)
    d[:5] = 0.0                       # the unshifted limit
    x[5:9] = F32(1.0)                 # the cube's far corner
    return x, w, nrm, d, g


@pytest.mark.parametrize("n", [4097, 3 * SMS * 128 + 77])
def test_shifted_fp32_forward_backward_and_disparity_gradient(n):
    """The FP32 engine in the shifted form: radiance to 1e-5 relative, table
    and decoder gradients and each query's dL/dd to 1e-5 normwise against
    the oracle (a ragged batch, and one of more than three tiles per CTA)."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    V = [17, 17, 9, 9, 5, 3]
    tree, ot = _tree(2100, 5, V)
    tables = I.make_tables(2101, tree.num_texels, 8, 0.3)
    weights = [W * F32(1.5) for W in I.make_mlp(2102, [48, 64, 64, 3])]
    sc = A.Scene(tree, dev(tables), [dev(W) for W in weights], device=DEV,
                 query_form=L.OCTA_FORM_SHIFTED)
    x, w, nrm, d, g = _queries(2103, n)
    X, Wd, Nd, Dd = dev(x), dev(w), dev(nrm), dev(d)
    rgb, _, addr = A.octa_query_fwd(sc, X, Wd, want_addr=True, normal=Nd, disparity=Dd)
    ref, enc = O.query_forward(ot, tables, weights, x, w, form="shifted", normal=nrm, disparity=d)
    np.testing.assert_array_equal(addr.cpu().numpy(), enc.addr.reshape(n, 6, 24))
    assert np.max(np.abs(rgb.cpu().numpy() / ref - 1)) <= 1e-5
    amb = decoder_ambiguous(weights, enc.h)
    d_rgb = g.normal(size=(n, 3)).astype(F32)
    d_rgb[amb] = 0.0
    dT = torch.zeros((tree.num_texels, 8), device=DEV)
    dW = torch.zeros(sc.weights.shape, device=DEV)
    dd = torch.full((n,), float("nan"), device=DEV)
    A.octa_query_bwd(sc, X, Wd, dev(d_rgb), [(dT, dW)], normal=Nd, disparity=Dd, d_disparity=dd)
    rT, rWs, _ = O.query_backward(ot, tables, weights, x, w, d_rgb, form="shifted", normal=nrm,
                                  disparity=d)
    rdd = O.disparity_gradient(ot, tables, weights, x, w, nrm, d, d_rgb)
    errs = [normwise(dT.cpu().numpy(), rT)] + weight_errors(dW.cpu().numpy(), rWs)
    e_dd = normwise(dd.cpu().numpy(), rdd)
    print(f"FP32 shifted backward ({int(amb.sum())} queries zeroed): tensors",
          [f"{e:.2e}" for e in errs], f"dL/dd {e_dd:.2e}")
    assert max(errs) <= 1e-5 and e_dd <= 1e-5


def test_shifted_bf16_disparity_gradient():
    """The tcgen05 backward's dL/dd (FP16 tables, BF16 decoder) against the
    oracle on the quantised parameters, within the BF16 path's bound for the
    gradients that flow through the ReLU masks (3 sqrt(f) + 1e-2, f the
    fraction of pre-activations within the BF16 forward error of zero); its
    table and decoder gradients unchanged by asking for dL/dd."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    V = [17, 17, 9, 9, 5, 3]
    tree, ot = _tree(2200, 5, V)
    tq = I.make_tables(2201, tree.num_texels, 8, 0.3).astype(np.float16).astype(F32)
    weights = [W * F32(1.5) for W in I.make_mlp(2202, [48, 64, 64, 3])]
    Wb = [dev(W).to(torch.bfloat16) for W in weights]
    wq = [W.float().cpu().numpy() for W in Wb]
    sc = A.Scene(tree, dev(tq).half().contiguous(), Wb, device=DEV, query_form=L.OCTA_FORM_SHIFTED)
    n = 20001
    x, w, nrm, d, g = _queries(2203, n)
    X, Wd, Nd, Dd = dev(x), dev(w), dev(nrm), dev(d)
    d_rgb = g.normal(size=(n, 3)).astype(F32)
    grads = []
    dd = torch.zeros(n, device=DEV)
    for want in (False, True):
        dT = torch.zeros((tree.num_texels, 8), device=DEV)
        dW = torch.zeros(sc.weights.shape, device=DEV)
        A.octa_query_bwd(sc, X, Wd, dev(d_rgb), [(dT, dW)], normal=Nd, disparity=Dd,
                         d_disparity=dd if want else None)
        grads.append((dT, dW))
    torch.cuda.synchronize()
    for a, b in zip(grads[0], grads[1]):
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) <= 1e-6
    rdd = O.disparity_gradient(ot, tq, wq, x, w, nrm, d, d_rgb)
    h = O.encode_features_shifted(ot, tq, x, w, nrm, d).h
    a, flags = h, []
    for W in [np.asarray(W, np.float64) for W in wq][:-1]:
        z = a @ W.T
        flags.append((np.abs(z) < 2.0 ** -7 * (np.abs(a) @ np.abs(W).T)).ravel())
        a = np.maximum(z, 0.0)
    frac = float(np.mean(np.concatenate(flags)))
    e = normwise(dd.cpu().numpy(), rdd)
    print("BF16 shifted dL/dd error", e, "mask fraction", frac)
    assert e <= 3.0 * np.sqrt(frac) + 1e-2


@pytest.mark.parametrize("levels,log2_T,n", [
    (8, 16, 3 * SMS * 128 + 5),   # dense first levels, hashed rest; > 3 tiles per CTA
    (4, 14, 1000),                # all dense
    (16, 12, 20001),              # hashed, many collisions, the widest input
])
def test_disparity_backward_matches_oracle(levels, log2_T, n):
    """octa_disparity_bwd (g_psi's backward, FP32) against the oracle's
    disparity_backward: hash-table and weight gradients to 1e-5 normwise;
    queries with an ambiguous g_psi mask carry no gradient."""
    from paper_2606_08469_gb300 import api as A
    res = O.hash_resolutions(levels, 16 if levels > 4 else 2, 512 if levels > 4 else 8)
    table, pw = I.predictor_params(2300 + levels, levels, log2_T, table_scale=0.3)
    pw = [W * F32(2.0) for W in pw]
    x, w, nrm, _, g = _queries(2310 + levels, n)
    c = g.normal(size=n).astype(F32)
    c[predictor_ambiguous(table, res, pw, x, w, nrm)] = 0.0
    pred = A.Predictor(table, res, pw, device=DEV)
    d_tab = torch.zeros(pred.table.shape, device=DEV)
    d_w = torch.zeros(pred.weights.shape, device=DEV)
    A.octa_disparity_bwd(pred, dev(x), dev(w), dev(nrm), dev(c), d_tab, d_w)
    rtab, rWs = O.disparity_backward(table, res, pw, x, w, nrm, c)
    errs = [normwise(d_tab.cpu().numpy(), rtab)] + weight_errors(d_w.cpu().numpy(), rWs)
    print(f"g_psi backward levels={levels}", [f"{e:.2e}" for e in errs])
    assert max(errs) <= 1e-5, errs


@pytest.mark.parametrize("levels,log2_T,n", [(8, 16, 3 * SMS * 256 + 33), (14, 12, 20001)])
def test_disparity_backward_tensor_cores(levels, log2_T, n):
    """octa_disparity_bwd on the tcgen05 path (the BF16 working copy of g_psi's
    weights given): hash-table and weight gradients against the oracle's
    disparity_backward on the BF16-rounded weights, within the BF16 path's
    bound for gradients behind ReLU masks (3 sqrt(f) + 1e-2, f the fraction of
    g_psi's hidden pre-activations within the BF16 forward error 2^-7 sum|w||a|
    of zero), the last layer's within 1e-2; more than three tiles per group
    slot and a ragged tail in the first case."""
    from paper_2606_08469_gb300 import api as A
    res = O.hash_resolutions(levels, 16, 512)
    table, pw = I.predictor_params(2350 + levels, levels, log2_T, table_scale=0.3)
    pw = [W * F32(2.0) for W in pw]
    x, w, nrm, _, g = _queries(2360 + levels, n)
    c = g.normal(size=n).astype(F32)
    pred = A.Predictor(table, res, pw, device=DEV, tensor_cores=True)
    pq = [W.astype(np.float32) for W in
          np.split(pred.weights_bf16.float().cpu().numpy(),
                   np.cumsum([W.size for W in pw])[:-1])]
    pq = [Wf.reshape(W.shape) for Wf, W in zip(pq, pw)]
    d_tab = torch.zeros(pred.table.shape, device=DEV)
    d_w = torch.zeros(pred.weights.shape, device=DEV)
    A.octa_disparity_bwd(pred, dev(x), dev(w), dev(nrm), dev(c), d_tab, d_w)
    rtab, rWs = O.disparity_backward(table, res, pq, x, w, nrm, c)
    inp = np.concatenate([O.hash_encode(table, res, x), O.reflect_f32(w, nrm).astype(np.float64)],
                         axis=1)
    a, flags = inp, []
    for W in [np.asarray(W, np.float64) for W in pq][:-1]:
        z = a @ W.T
        flags.append((np.abs(z) < 2.0 ** -7 * (np.abs(a) @ np.abs(W).T)).ravel())
        a = np.maximum(z, 0.0)
    frac = float(np.mean(np.concatenate(flags)))
    errs = [normwise(d_tab.cpu().numpy(), rtab)] + weight_errors(d_w.cpu().numpy(), rWs)
    bound = 3.0 * np.sqrt(frac) + 1e-2
    print(f"tensor-core g_psi backward levels={levels}", [f"{e:.2e}" for e in errs],
          "mask fraction", round(frac, 5), "bound", round(bound, 4))
    assert errs[-1] <= 1e-2 and max(errs) <= bound


def _step_inputs(n_pairs, seed=2400):
    """A shifted-form training batch: depth-5 tree with vertex maps, F = 8
    FP32 tables, decoder 48-64-64-3, an 8-level g_psi, pairs with normals."""
    V = [17, 17, 9, 9, 5, 3]
    tree, ot = _tree(seed, 5, V)
    tables = I.make_tables(seed + 1, tree.num_texels, 8, 0.3)
    weights = [W * F32(1.5) for W in I.make_mlp(seed + 2, [48, 64, 64, 3])]
    levels = 8
    res = O.hash_resolutions(levels, 16, 512)
    ptab, pw = I.predictor_params(seed + 3, levels, 16, table_scale=0.3)
    pw = [W * F32(2.0) for W in pw]
    pairs, n1, n2 = I.training_pairs_with_normals(seed + 4, n_pairs)
    return tree, ot, tables, weights, (ptab, res, pw), pairs, n1, n2


def _neutralised(ot, tables, weights, pred, pairs, n1, n2):
    """The batch with every pair that has an ambiguous decision given a zero
    residual (module docstring); returns it and the count."""
    ptab, res, pw = pred
    n = pairs.n
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    Nr = np.concatenate([n1, n2])
    d32 = O.disparity(ptab, res, pw, X, Om, Nr).astype(F32)
    rgb, enc = O.query_forward(ot, tables, weights, X, Om, form="shifted", normal=Nr,
                               disparity=d32)
    bad = decoder_ambiguous(weights, enc.h) | predictor_ambiguous(ptab, res, pw, X, Om, Nr)
    bad |= lookup_unstable(ot, tables, X, Om, Nr, d32)
    bad = bad[:n] | bad[n:]
    return neutralise_pairs(pairs, bad, rgb[:n]), int(bad.sum())


@pytest.mark.parametrize("rhs_grad", [True, False])
def test_shifted_fused_pass_fp32(rhs_grad):
    """octa_train_fused in the shifted form on the FP32 engine, the
    disparities given: loss, table and decoder gradients and both queries'
    dL/dd to 1e-5 against the oracle."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    tree, ot, tables, weights, pred, pairs, n1, n2 = _step_inputs(6001)
    n = pairs.n
    g = I.rng(2450)
    d1 = g.uniform(0.0, 6.0, n).astype(F32)
    d2 = g.uniform(0.0, 6.0, n).astype(F32)
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    Nr = np.concatenate([n1, n2])
    D = np.concatenate([d1, d2])
    rgb, enc = O.query_forward(ot, tables, weights, X, Om, form="shifted", normal=Nr, disparity=D)
    bad = decoder_ambiguous(weights, enc.h)
    pairs = neutralise_pairs(pairs, bad[:n] | bad[n:], rgb[:n])
    sc = A.Scene(tree, dev(tables), [dev(W) for W in weights], device=DEV,
                 query_form=L.OCTA_FORM_SHIFTED)
    dT = torch.zeros((tree.num_texels, 8), device=DEV)
    dW = torch.zeros(sc.weights.shape, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    dd1 = torch.zeros(n, device=DEV)
    dd2 = torch.zeros(n, device=DEV)
    # octa_pairs.omega2 is the secondary query's direction itself, -omega'
    A.octa_train_fused(sc, dev(pairs.x), dev(pairs.omega), dev(pairs.x2), dev(-pairs.omega2),
                       dev(pairs.E), dev(pairs.w), [(dT, dW)], loss, rhs_grad=rhs_grad,
                       shift=(dev(n1), dev(n2), dev(d1), dev(d2), dd1, dd2))
    rl, dLp, dLs = O.residual_loss(rgb[:n], rgb[n:], pairs.E, pairs.w, rhs_grad=rhs_grad)
    d_rgb = np.concatenate([dLp, dLs])
    rT, rWs, _ = O.query_backward(ot, tables, weights, X, Om, d_rgb, form="shifted", normal=Nr,
                                  disparity=D)
    rdd = O.disparity_gradient(ot, tables, weights, X, Om, Nr, D, d_rgb)
    assert abs(loss.item() - rl) <= 1e-5 * rl
    errs = [normwise(dT.cpu().numpy(), rT)] + weight_errors(dW.cpu().numpy(), rWs)
    gdd = np.concatenate([dd1.cpu().numpy(), dd2.cpu().numpy()])
    e_dd = normwise(gdd, rdd)
    if not rhs_grad:
        assert np.all(gdd[n:] == 0.0)      # the target is detached: no secondary gradient
    print("FP32 shifted fused pass", [f"{e:.2e}" for e in errs], f"dL/dd {e_dd:.2e}")
    assert max(errs) <= 1e-5 and e_dd <= 1e-5


def test_shifted_fused_pass_bf16_equals_unfused():
    """The tcgen05 fused pass in the shifted form against the same kernel's
    unfused passes (octa_query_fwd, residual_loss's formulas, octa_query_bwd)
    on the same inputs: loss, gradients and dL/dd agree to FP32 rounding
    (atomics order), so the fused pass routes both queries' inputs and
    outputs right; the unfused passes are checked against the oracle above."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    tree, ot, tables, weights, pred, pairs, n1, n2 = _step_inputs(9001, seed=2500)
    n = pairs.n
    g = I.rng(2550)
    d1 = g.uniform(0.0, 6.0, n).astype(F32)
    d2 = g.uniform(0.0, 6.0, n).astype(F32)
    Wb = [dev(W).to(torch.bfloat16) for W in weights]
    sc = A.Scene(tree, dev(tables).half().contiguous(), Wb, device=DEV,
                 query_form=L.OCTA_FORM_SHIFTED)
    P = {k: dev(getattr(pairs, k)) for k in ("x", "omega", "x2", "omega2", "E", "w")}
    N1, N2, D1, D2 = dev(n1), dev(n2), dev(d1), dev(d2)
    dT = torch.zeros((tree.num_texels, 8), device=DEV)
    dW = torch.zeros(sc.weights.shape, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    dd1 = torch.zeros(n, device=DEV)
    dd2 = torch.zeros(n, device=DEV)
    A.octa_train_fused(sc, P["x"], P["omega"], P["x2"], -P["omega2"], P["E"], P["w"], [(dT, dW)],
                       loss, shift=(N1, N2, D1, D2, dd1, dd2))
    X = torch.cat([P["x"], P["x2"]])
    Om = torch.cat([P["omega"], -P["omega2"]])
    Nr, D = torch.cat([N1, N2]), torch.cat([D1, D2])
    rgb, _, _ = A.octa_query_fwd(sc, X, Om, normal=Nr, disparity=D)
    Lp, Ls = rgb[:n].double(), rgb[n:].double()
    T = P["E"].double() + P["w"].double() * Ls
    den = Lp + T + 1e-2
    r = (Lp - T) / den
    rl = float((r * r).sum() / (3 * n))
    dLp = (2.0 * r / (3 * n * den)).float()
    dLs = (-2.0 * r * P["w"].double() / (3 * n * den)).float()
    uT = torch.zeros_like(dT)
    uW = torch.zeros_like(dW)
    udd = torch.zeros(2 * n, device=DEV)
    A.octa_query_bwd(sc, X, Om, torch.cat([dLp, dLs]), [(uT, uW)], normal=Nr, disparity=D,
                     d_disparity=udd)
    torch.cuda.synchronize()
    e = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    print("BF16 shifted fused vs unfused: loss", abs(loss.item() - rl) / rl, "tables", e(dT, uT),
          "weights", e(dW, uW), "dL/dd", e(torch.cat([dd1, dd2]), udd))
    assert abs(loss.item() - rl) <= 1e-5 * rl
    assert e(dT, uT) <= 1e-3 and e(dW, uW) <= 1e-3 and e(torch.cat([dd1, dd2]), udd) <= 1e-3


def test_shifted_whole_step_fp32():
    """The paper's full model trained for one step on the GPU (FP32): d =
    g_psi(x, omega_r) for every primary and secondary query (octa_disparity),
    the fused shifted pass with both queries' dL/dd (octa_train_fused), g_psi's
    backward (octa_disparity_bwd), then Adam over the four parameter groups
    (adam_step): the loss, the decoder, table, hash-table and g_psi weight
    gradients to 1e-5 and the updated parameters against the oracle's
    shifted_train_gradients and Adam (with more tiles than one per CTA)."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    tree, ot, tables, weights, pred, pairs, n1, n2 = _step_inputs(3 * SMS * 64 + 13, seed=2600)
    ptab, res, pw = pred
    pairs, n_bad = _neutralised(ot, tables, weights, pred, pairs, n1, n2)
    n = pairs.n
    assert n_bad < n // 10
    sc = A.Scene(tree, dev(tables), [dev(W) for W in weights], device=DEV,
                 query_form=L.OCTA_FORM_SHIFTED)
    gp = A.Predictor(ptab, res, pw, device=DEV)
    P = {k: dev(getattr(pairs, k)) for k in ("x", "omega", "x2", "omega2", "E", "w")}
    N1, N2 = dev(n1), dev(n2)
    S = 2.0 ** 10
    scaler = A.make_scaler(S, growth_interval=0, device=DEV)
    d1 = A.octa_disparity(gp, P["x"], P["omega"], N1)
    d2 = A.octa_disparity(gp, P["x2"], -P["omega2"], N2)
    dT = torch.zeros((tree.num_texels, 8), device=DEV)
    dW = torch.zeros(sc.weights.shape, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    dd1 = torch.zeros(n, device=DEV)
    dd2 = torch.zeros(n, device=DEV)
    A.octa_train_fused(sc, P["x"], P["omega"], P["x2"], -P["omega2"], P["E"], P["w"], [(dT, dW)],
                       loss, scaler=scaler, shift=(N1, N2, d1, d2, dd1, dd2))
    d_tab = torch.zeros(gp.table.shape, device=DEV)
    d_pw = torch.zeros(gp.weights.shape, device=DEV)
    A.octa_disparity_bwd(gp, torch.cat([P["x"], P["x2"]]), torch.cat([P["omega"], -P["omega2"]]),
                         torch.cat([N1, N2]), torch.cat([dd1, dd2]), d_tab, d_pw)
    torch.cuda.synchronize()
    rl, rT, rWs, rtab, rWp, rdd, rd = O.shifted_train_gradients(ot, tables, weights, pred, pairs,
                                                                n1, n2, scale=S)
    d_gpu = torch.cat([d1, d2]).cpu().numpy()
    assert np.max(np.abs(d_gpu / rd - 1)) <= 1e-5
    assert abs(loss.item() - rl) <= 1e-5 * rl
    errs = {"tables": normwise(dT.cpu().numpy(), rT),
            "decoder": max(weight_errors(dW.cpu().numpy(), rWs)),
            "dL/dd": normwise(torch.cat([dd1, dd2]).cpu().numpy(), rdd),
            "hash tables": normwise(d_tab.cpu().numpy(), rtab),
            "g_psi": max(weight_errors(d_pw.cpu().numpy(), rWp))}
    print(f"whole shifted step ({n_bad} pairs zeroed)", {k: f"{v:.2e}" for k, v in errs.items()})
    assert max(errs.values()) <= 1e-5, errs
    # Adam over the four groups (tables and g_psi lr 1e-2, MLPs 1e-3)
    groups, masters = [], []
    for param, grad, lr in ((sc.tables, dT, 1e-2), (sc.weights, dW, 1e-3),
                            (gp.table.reshape(-1), d_tab.reshape(-1), 1e-2),
                            (gp.weights, d_pw, 1e-3)):
        p32 = param.reshape(-1).clone()
        masters.append(p32)
        groups.append(A.ParamGroup(p32, grad.reshape(-1), torch.zeros_like(p32),
                                   torch.zeros_like(p32), lr))
    ws = A.workspace(L.OCTA_OP_ADAM, sum(int(m.numel()) for m in masters), device=DEV)
    A.adam_step(groups, scaler, ws)
    torch.cuda.synchronize()
    refs = [(tables.ravel(), rT.ravel(), 1e-2),
            (np.concatenate([W.ravel() for W in weights]), np.concatenate([g.ravel() for g in rWs]),
             1e-3),
            (ptab.ravel(), rtab.ravel(), 1e-2),
            (np.concatenate([W.ravel() for W in pw]), np.concatenate([g.ravel() for g in rWp]),
             1e-3)]
    for m, (p0, gr, lr) in zip(masters, refs):
        want, _, _ = O.adam_update(p0, gr / S, np.zeros_like(p0, np.float64),
                                   np.zeros_like(p0, np.float64), 1, lr)
        got = m.cpu().numpy()
        # the first Adam step moves every touched parameter by lr g / (|g| + eps):
        # compare the updates normwise
        upd, ref_upd = got - p0, want - p0
        assert normwise(upd, ref_upd) <= 1e-3, normwise(upd, ref_upd)


def test_shifted_train_step_wrapper_and_graph():
    """train.ShiftedTrainStep (g_psi forward, fused shifted pass, g_psi
    backward, Adam over four groups) on train_f32's scene with vertex maps:
    its gradients before Adam against the oracle's shifted_train_gradients
    (1e-3 normwise: no pairs are neutralised here, the strict comparison is
    test_shifted_whole_step_fp32), and a CUDA-graph replay of three steps
    against three eager steps of a second, identical instance."""
    from paper_2606_08469_gb300 import inputs as I
    from paper_2606_08469_gb300 import workloads as WL
    cfg = I.WORKLOADS["train_f32"]
    a, (tree, tables, weights, pred, pairs, n1, n2) = WL.shifted_train_step_for(
        cfg, n_pairs=4096, device=DEV, precision="f32")
    ot = O.build_tree(cfg.seed("tree"), cfg.max_depth, cfg.p_base, [r + 1 for r in cfg.R])
    a.predict()
    a.fused_pass()
    a.predictor_backward()
    torch.cuda.synchronize()
    S = 2.0 ** 15
    rl, rT, rWs, rtab, rWp, _, _ = O.shifted_train_gradients(ot, tables, weights, pred, pairs,
                                                             n1, n2, scale=S)
    assert abs(a.loss.item() - rl) <= 1e-5 * rl
    errs = [normwise(a.state.grad_t.cpu().numpy(), rT),
            max(weight_errors(a.state.grad_w.cpu().numpy(), rWs)),
            normwise(a.pred_state.grad_t.cpu().numpy(), rtab),
            max(weight_errors(a.pred_state.grad_w.cpu().numpy(), rWp))]
    print("ShiftedTrainStep gradients vs FP64", [f"{e:.2e}" for e in errs])
    assert max(errs) <= 1e-3
    a.optimizer()
    for _ in range(2):
        a.step()
    b, _ = WL.shifted_train_step_for(cfg, n_pairs=4096, device=DEV, precision="f32")
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        b.step(stream)                       # eager warm-up: step 1
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            b.step(stream)
        g.replay()                           # steps 2, 3
        g.replay()
    stream.synchronize()
    torch.cuda.synchronize()
    e = lambda u, v: float(torch.linalg.norm(u - v) / torch.linalg.norm(v))
    for u, v in ((a.state.master_t, b.state.master_t), (a.state.master_w, b.state.master_w),
                 (a.pred_state.pred.table, b.pred_state.pred.table),
                 (a.pred_state.pred.weights, b.pred_state.pred.weights)):
        assert e(u, v) <= 1e-6, e(u, v)


def test_training_entry_point_errors():
    """Refusals of the new arguments: d_disparity outside the shifted form,
    the shifted fused pass without the secondaries' inputs, the one-launch
    step in the shifted form, and octa_disparity_bwd with missing arrays or
    more than 14 levels on the tensor cores; an empty batch does nothing."""
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    V = [5, 5, 3]
    tree = A.octree_build(2700, 2, 0.8, V)
    tables = I.make_tables(2701, tree.num_texels, 8, 0.3)
    weights = [dev(W) for W in I.make_mlp(2702, [24, 64, 64, 3])]
    cell = A.Scene(tree, dev(tables), weights, device=DEV)
    sh = A.Scene(tree, dev(tables), weights, device=DEV, query_form=L.OCTA_FORM_SHIFTED)
    x, w, nrm, d, g = _queries(2703, 300)
    X, Wd, Nd, Dd = dev(x), dev(w), dev(nrm), dev(d)
    d_rgb = dev(g.normal(size=(300, 3)).astype(F32))
    dT = torch.zeros((tree.num_texels, 8), device=DEV)
    dW = torch.zeros(cell.weights.shape, device=DEV)
    dd = torch.zeros(300, device=DEV)
    with pytest.raises(L.OctaError) as e:
        A.octa_query_bwd(cell, X, Wd, d_rgb, [(dT, dW)], d_disparity=dd)
    assert e.value.code == L.OCTA_EINVAL
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    E = torch.zeros((300, 3), device=DEV)
    with pytest.raises(L.OctaError) as e:      # no normal2 / disparity2
        A.octa_train_fused(sh, X, Wd, X, -Wd, E, E, [(dT, dW)], loss,
                           shift=(Nd, None, Dd, None, None, None))
    assert e.value.code == L.OCTA_EINVAL
    scaler = A.make_scaler(device=DEV)
    ws = A.workspace(L.OCTA_OP_STEP, 0, device=DEV)
    groups = [A.ParamGroup(dT.reshape(-1).clone(), dT.reshape(-1), torch.zeros_like(dT).reshape(-1),
                           torch.zeros_like(dT).reshape(-1), 1e-2)]
    with pytest.raises(L.OctaError) as e:      # the one-launch step: no shifted form
        A.octa_train_step_batched(sh, X, Wd, X, -Wd, E, E, [(dT, dW)], groups, loss, scaler, ws)
    assert e.value.code == L.OCTA_EUNSUPPORTED
    table, pw = I.predictor_params(2704, 15, 10)
    res = O.hash_resolutions(15, 4, 64)
    pred = A.Predictor(table, res, pw, device=DEV, tensor_cores=True)
    d_tab = torch.zeros(pred.table.shape, device=DEV)
    d_w = torch.zeros(pred.weights.shape, device=DEV)
    with pytest.raises(L.OctaError) as e:      # 15 levels on the tensor cores
        A.octa_disparity_bwd(pred, X, Wd, Nd, dd, d_tab, d_w)
    assert e.value.code == L.OCTA_ERANGE
    pred32 = A.Predictor(table, res, pw, device=DEV)
    q = A._queries(X, Wd, None)                # no normal
    with pytest.raises(L.OctaError) as e:
        L.check(A._lib().octa_disparity_bwd(A.C.byref(pred32.as_c()), A.C.byref(q),
                                            A._ptr(dd), A._ptr(d_tab), A._ptr(d_w),
                                            A._stream()), "octa_disparity_bwd")
    assert e.value.code == L.OCTA_EINVAL
    A.octa_disparity_bwd(pred32, X[:0], Wd[:0], Nd[:0], dd[:0], d_tab, d_w)
    torch.cuda.synchronize()
    assert float(d_tab.abs().sum()) == 0.0 and float(d_w.abs().sum()) == 0.0
