"""One neural-radiosity training step through the C ABI.

A step queries L_hat at every primary (x, omega) and secondary (x', -omega')
(Eq. 2 gives the sign), evaluates the Eq. 14 residual against the one-sample
target of Eq. 3, back-propagates into the feature tables and the decoder and
applies Adam with dynamic loss scaling.  Each of these is one library call on
the caller's stream; the sequence can be captured in a CUDA graph.
"""
from __future__ import annotations

import torch

from . import _lib as L
from . import api


class SceneState:
    """Master parameters, gradients, Adam moments and working copies of one scene."""

    def __init__(self, tree, tables, weights, table_dtype, weight_dtype, device, query_form=0):
        dev = torch.device(device)
        self.master_t = torch.as_tensor(tables, dtype=torch.float32).to(dev).contiguous()
        self.master_w = torch.cat([torch.as_tensor(W, dtype=torch.float32).reshape(-1)
                                   for W in weights]).to(dev).contiguous()
        self.grad_t = torch.zeros_like(self.master_t)
        self.grad_w = torch.zeros_like(self.master_w)
        self.m_t = torch.zeros_like(self.master_t)
        self.v_t = torch.zeros_like(self.master_t)
        self.m_w = torch.zeros_like(self.master_w)
        self.v_w = torch.zeros_like(self.master_w)
        self.work_t = None if table_dtype == torch.float32 else self.master_t.to(table_dtype)
        self.work_w = None if weight_dtype == torch.float32 else self.master_w.to(weight_dtype)
        shaped = [torch.empty(W.shape) for W in weights]
        self.scene = api.Scene(tree, self.work_t if self.work_t is not None else self.master_t,
                               shaped, device=dev, query_form=query_form)
        self.scene.set_weights_flat(self.work_w if self.work_w is not None else self.master_w)

    def groups(self, lr_tables, lr_mlp):
        return [api.ParamGroup(self.master_t, self.grad_t, self.m_t, self.v_t, lr_tables, self.work_t),
                api.ParamGroup(self.master_w, self.grad_w, self.m_w, self.v_w, lr_mlp, self.work_w)]


class TrainStep:
    """Training step over one or several scenes (queries ordered scene by
    scene, each scene's primaries followed by its secondaries)."""

    def __init__(self, scene_states, pairs, eps=1e-2, rhs_grad=True, lr_tables=1e-2, lr_mlp=1e-3,
                 scale=2.0 ** 15, growth_interval=2000, device="cuda", fused=False,
                 persistent=False, norm_pairs=None):
        dev = torch.device(device)
        self.states = scene_states
        self.scenes = [s.scene for s in scene_states]
        self.n = [int(p["x"].shape[0]) for p in pairs]
        xs, oms, Es, ws = [], [], [], []
        for p in pairs:
            xs += [p["x"], p["x2"]]
            oms += [p["omega"], -p["omega2"]]
            Es.append(p["E"])
            ws.append(p["w"])
        self.X = torch.cat(xs).to(dev).contiguous()
        self.Om = torch.cat(oms).to(dev).contiguous()
        self.E = [e.to(dev).contiguous() for e in Es]
        self.w = [w.to(dev).contiguous() for w in ws]
        self.counts = [2 * n for n in self.n]
        total = sum(self.counts)
        self.rgb = torch.empty((total, 3), dtype=torch.float32, device=dev)
        self.d_rgb = torch.zeros((total, 3), dtype=torch.float32, device=dev)
        self.loss = torch.zeros(len(self.n), dtype=torch.float64, device=dev)
        self.scaler = api.make_scaler(scale, growth_interval, device=dev)
        self.ws_loss = api.workspace(L.OCTA_OP_LOSS, max(self.n), device=dev)
        self.ws_adam = api.workspace(L.OCTA_OP_ADAM, 0, device=dev)
        self.eps, self.rhs_grad = eps, rhs_grad
        self.lr_tables, self.lr_mlp = lr_tables, lr_mlp
        self.groups = [g for s in scene_states for g in s.groups(lr_tables, lr_mlp)]
        self.grads = [(s.grad_t, s.grad_w) for s in scene_states]
        # fused mode: one octa_train_fused launch replaces forward + loss +
        # backward; the pair arrays are kept per role
        # persistent mode: the fused pass and Adam in one cooperative launch
        self.persistent = persistent
        self.fused = fused or persistent
        # pairs each scene's loss is a mean over (None: the scene's own pairs;
        # a data-parallel shard passes the whole batch's counts)
        self.norm_pairs = None if norm_pairs is None else [int(m) for m in norm_pairs]
        if self.norm_pairs is not None and not self.fused:
            raise ValueError("norm_pairs needs the fused training pass")
        if persistent:
            self.ws_step = api.workspace(L.OCTA_OP_STEP, 0, device=dev)
        if self.fused:
            cat = lambda k: torch.cat([p[k] for p in pairs]).to(dev).contiguous()
            self.Px, self.Pw, self.Sx = cat("x"), cat("omega"), cat("x2")
            self.Sw = torch.cat([-p["omega2"] for p in pairs]).to(dev).contiguous()
            self.Ecat, self.wcat = cat("E"), cat("w")

    def use_flat_gradients(self, extra=0):
        """Move every scene's gradient buffers into one flat FP32 tensor (each
        buffer at a 16-byte aligned offset, as the float4 scatter needs) with
        `extra` free slots at its end, and point the kernels' gradient
        arguments and Adam's groups at the views.  Returns the flat tensor
        (a data-parallel step all-reduces it with one collective)."""
        sizes = []
        for s in self.states:
            sizes += [s.grad_t.numel(), s.grad_w.numel()]
        offs, off = [], 0
        for n in sizes:
            offs.append(off)
            off += (n + 3) // 4 * 4
        flat = torch.zeros(off + extra, dtype=torch.float32, device=self.states[0].grad_t.device)
        k = 0
        for s in self.states:
            for name in ("grad_t", "grad_w"):
                old = getattr(s, name)
                view = flat[offs[k]:offs[k] + old.numel()].view(old.shape)
                view.copy_(old)
                setattr(s, name, view)
                k += 1
        self.groups = [g for s in self.states for g in s.groups(self.lr_tables, self.lr_mlp)]
        self.grads = [(s.grad_t, s.grad_w) for s in self.states]
        self.flat_grads = flat
        return flat

    PAIR_INPUTS = ("Px", "Pw", "Sx", "Sw", "Ecat", "wcat")

    def pair_inputs(self):
        """The device arrays the fused pass reads (primaries, secondaries,
        emission, BSDF weight), by name."""
        return {k: getattr(self, k) for k in self.PAIR_INPUTS}

    def set_pair_inputs(self, arrays):
        """Point the fused pass at other device arrays of the same shapes
        (double-buffered input copies)."""
        for k in self.PAIR_INPUTS:
            t = arrays[k]
            cur = getattr(self, k)
            if t.shape != cur.shape or t.dtype != cur.dtype or t.device != cur.device:
                raise ValueError(f"{k}: expected {tuple(cur.shape)} {cur.dtype} on {cur.device}")
            setattr(self, k, t)

    def forward(self, stream=None):
        api.octa_query_fwd(self.scenes, self.X, self.Om, self.counts, rgb=self.rgb, stream=stream)

    def loss_and_grad(self, stream=None):
        off = 0
        for s, n in enumerate(self.n):
            api.residual_loss(self.rgb[off:off + n], self.rgb[off + n:off + 2 * n], self.E[s],
                              self.w[s], self.d_rgb[off:off + n], self.d_rgb[off + n:off + 2 * n],
                              self.loss[s:s + 1], self.ws_loss, self.eps, self.rhs_grad,
                              self.scaler, stream=stream)
            off += 2 * n

    def backward(self, stream=None):
        api.octa_query_bwd(self.scenes, self.X, self.Om, self.d_rgb, self.grads, self.counts,
                           stream=stream)

    def optimizer(self, stream=None):
        api.adam_step(self.groups, self.scaler, self.ws_adam, stream=stream)

    def fused_pass(self, stream=None):
        api.octa_train_fused(self.scenes, self.Px, self.Pw, self.Sx, self.Sw, self.Ecat, self.wcat,
                             self.grads, self.loss, self.n, self.eps, self.rhs_grad, self.scaler,
                             stream=stream, norm_pairs=self.norm_pairs)

    def persistent_step(self, stream=None, status=None, timeout_ns=0, extra_arrivals=0,
                        skip_first_mma=0):
        api.octa_train_step_batched(self.scenes, self.Px, self.Pw, self.Sx, self.Sw, self.Ecat,
                                    self.wcat, self.grads, self.groups, self.loss, self.scaler,
                                    self.ws_step, self.n, self.eps, self.rhs_grad,
                                    timeout_ns=timeout_ns, extra_arrivals=extra_arrivals,
                                    status=status, stream=stream, norm_pairs=self.norm_pairs,
                                    skip_first_mma=skip_first_mma)

    def step(self, stream=None):
        if self.persistent:
            self.persistent_step(stream)
            return
        if self.fused:
            self.fused_pass(stream)
        else:
            self.forward(stream)
            self.loss_and_grad(stream)
            self.backward(stream)
        self.optimizer(stream)


def quarter_schedule(step, total_steps, n0, m0, quarters=4):
    """(LHS samples, RHS samples M) of 0-based step `step` of `total_steps`:
    the LHS count halves and M doubles after every quarter (Section 4)."""
    if total_steps < 1 or step < 0:
        raise ValueError("need total_steps >= 1 and step >= 0")
    q = min(quarters - 1, (quarters * step) // total_steps)
    return n0 >> q, m0 << q


class MultiSampleStep:
    """Training step of Section 4's regime on one scene: every LHS sample
    (x, omega) is supervised by Eq. 3's target over M RHS samples.

    Per step, all through the C ABI: octa_trace_rays finds the secondary
    hits x'^m of the N*M sampled directions (Eq. 2) and writes them, with
    the query directions -omega_i^m, after the N primaries; one
    octa_query_fwd evaluates the N + N*M queries; residual_loss_multi forms
    the target and Eq. 14; octa_query_bwd back-propagates the primaries
    (and, with rhs_grad, the secondaries); adam_step updates.
    samples: dict of device tensors x [N][3], omega [N][3], E [N][3],
    omega_i [N][M][3], w [N][M][3]; prims: api.Prims of the scene."""

    def __init__(self, state, prims, samples, eps=1e-2, rhs_grad=False, lr_tables=1e-2,
                 lr_mlp=1e-3, scale=2.0 ** 15, growth_interval=2000, t_min=1e-4, device="cuda"):
        dev = torch.device(device)
        self.state, self.scene, self.prims = state, state.scene, prims
        N, M = int(samples["omega_i"].shape[0]), int(samples["omega_i"].shape[1])
        self.N, self.M = N, M
        total = N + N * M
        self.X = torch.empty((total, 3), dtype=torch.float32, device=dev)
        self.Om = torch.empty((total, 3), dtype=torch.float32, device=dev)
        self.X[:N].copy_(samples["x"])
        self.Om[:N].copy_(samples["omega"])
        self.dirs = samples["omega_i"].reshape(N * M, 3).to(dev).contiguous()
        self.E = samples["E"].to(dev).contiguous()
        self.w = samples["w"].to(dev).contiguous()
        self.rgb = torch.empty((total, 3), dtype=torch.float32, device=dev)
        self.d_rgb = torch.zeros((total, 3), dtype=torch.float32, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.scaler = api.make_scaler(scale, growth_interval, device=dev)
        self.ws_loss = api.workspace(L.OCTA_OP_LOSS, N, device=dev)
        self.ws_adam = api.workspace(L.OCTA_OP_ADAM, 0, device=dev)
        self.eps, self.rhs_grad, self.t_min = eps, rhs_grad, t_min
        self.groups = state.groups(lr_tables, lr_mlp)
        self.grads = [(state.grad_t, state.grad_w)]

    @property
    def queries_per_step(self):
        return self.N * (1 + self.M)

    def trace(self, stream=None):
        N = self.N
        api.octa_trace_rays(self.prims, self.X[:N], self.dirs, self.M, self.t_min,
                            hit=self.X[N:], query_dir=self.Om[N:], stream=stream)

    def forward(self, stream=None):
        api.octa_query_fwd(self.scene, self.X, self.Om, rgb=self.rgb, stream=stream)

    def loss_and_grad(self, stream=None):
        N, M = self.N, self.M
        api.residual_loss_multi(self.rgb[:N], self.rgb[N:].view(N, M, 3), self.E, self.w,
                                self.d_rgb[:N], self.d_rgb[N:].view(N, M, 3), self.loss,
                                self.ws_loss, self.eps, self.rhs_grad, self.scaler, stream=stream)

    def backward(self, stream=None):
        if self.rhs_grad:
            api.octa_query_bwd(self.scene, self.X, self.Om, self.d_rgb, self.grads, stream=stream)
        else:  # the target is detached: only the primaries carry gradient
            N = self.N
            api.octa_query_bwd(self.scene, self.X[:N], self.Om[:N], self.d_rgb[:N], self.grads,
                               stream=stream)

    def optimizer(self, stream=None):
        api.adam_step(self.groups, self.scaler, self.ws_adam, stream=stream)

    def step(self, stream=None):
        self.trace(stream)
        self.forward(stream)
        self.loss_and_grad(stream)
        self.backward(stream)
        self.optimizer(stream)


class PredictorState:
    """Master parameters, gradients and Adam moments of the disparity
    predictor g_psi (hash tables [L][T][2] and its MLP), FP32; with
    tensor_cores its forward runs on the tcgen05 path from a BF16 working
    copy of the weights that Adam refreshes."""

    def __init__(self, table, res, weights, device, tensor_cores=False):
        self.pred = api.Predictor(table, res, weights, device=device, tensor_cores=tensor_cores)
        self.grad_t = torch.zeros_like(self.pred.table)
        self.grad_w = torch.zeros_like(self.pred.weights)
        self.m_t = torch.zeros_like(self.pred.table)
        self.v_t = torch.zeros_like(self.pred.table)
        self.m_w = torch.zeros_like(self.pred.weights)
        self.v_w = torch.zeros_like(self.pred.weights)

    def groups(self, lr_table, lr_mlp):
        flat = lambda t: t.reshape(-1)
        return [api.ParamGroup(flat(self.pred.table), flat(self.grad_t), flat(self.m_t),
                               flat(self.v_t), lr_table),
                api.ParamGroup(self.pred.weights, self.grad_w, self.m_w, self.v_w, lr_mlp,
                               self.pred.weights_bf16)]


class ShiftedTrainStep:
    """A training step of the paper's full model on one scene (Eq. 7-9,
    Eq. 14; Section 3.3: the disparity is learnt only through the radiance
    objective).  Per step, all through the C ABI on the caller's stream:
    octa_disparity predicts d = g_psi(x, omega_r) for the N primaries and N
    secondaries in one launch; octa_train_fused runs the shifted lookup, the
    decoder, the Eq. 14 gradient and the backward of every pair and returns
    each query's dL/dd; octa_disparity_bwd carries dL/dd into g_psi's hash
    tables and weights; adam_step updates the four parameter groups (tables,
    decoder, hash tables, g_psi's MLP).  The scene state must be in the
    shifted form; pairs: dict of device tensors x, omega, x2, omega2, E, w
    (omega2 the sampled incident direction omega') and normal, normal2."""

    def __init__(self, state, pred_state, pairs, eps=1e-2, rhs_grad=True, lr_tables=1e-2,
                 lr_mlp=1e-3, lr_hash=1e-2, lr_pred=1e-3, scale=2.0 ** 15, growth_interval=2000,
                 device="cuda"):
        dev = torch.device(device)
        self.state, self.pred_state = state, pred_state
        self.scene = state.scene
        n = int(pairs["x"].shape[0])
        self.n = n
        cat = lambda a, b: torch.cat([a, b]).to(dev).contiguous()
        self.X = cat(pairs["x"], pairs["x2"])
        self.Om = cat(pairs["omega"], -pairs["omega2"])
        self.Nr = cat(pairs["normal"], pairs["normal2"])
        self.E = pairs["E"].to(dev).contiguous()
        self.w = pairs["w"].to(dev).contiguous()
        self.D = torch.empty(2 * n, dtype=torch.float32, device=dev)
        self.dD = torch.zeros(2 * n, dtype=torch.float32, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.scaler = api.make_scaler(scale, growth_interval, device=dev)
        self.ws_adam = api.workspace(L.OCTA_OP_ADAM, 0, device=dev)
        self.eps, self.rhs_grad = eps, rhs_grad
        self.groups = state.groups(lr_tables, lr_mlp) + pred_state.groups(lr_hash, lr_pred)
        self.grads = [(state.grad_t, state.grad_w)]

    def predict(self, stream=None):
        api.octa_disparity(self.pred_state.pred, self.X, self.Om, self.Nr, out=self.D,
                           stream=stream)

    def fused_pass(self, stream=None):
        n = self.n
        api.octa_train_fused(self.scene, self.X[:n], self.Om[:n], self.X[n:], self.Om[n:],
                             self.E, self.w, self.grads, self.loss, None, self.eps, self.rhs_grad,
                             self.scaler, stream=stream,
                             shift=(self.Nr[:n], self.Nr[n:], self.D[:n], self.D[n:],
                                    self.dD[:n], self.dD[n:]))

    def predictor_backward(self, stream=None):
        ps = self.pred_state
        api.octa_disparity_bwd(ps.pred, self.X, self.Om, self.Nr, self.dD, ps.grad_t, ps.grad_w,
                               stream=stream)

    def optimizer(self, stream=None):
        api.adam_step(self.groups, self.scaler, self.ws_adam, stream=stream)

    def step(self, stream=None):
        self.predict(stream)
        self.fused_pass(stream)
        self.predictor_backward(stream)
        self.optimizer(stream)
