"""Thin torch-facing binding of the C ABI: argument marshalling only.

Every computation runs in the CUDA library; this module only turns torch
tensors (device memory) and the current torch stream into the ABI's plain
pointers, sizes and structs.  Function names follow the header.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L

_DT = {torch.float32: L.OCTA_F32, torch.float16: L.OCTA_F16, torch.bfloat16: L.OCTA_BF16}


def _lib():
    return L.load()


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# octree (host)
# ---------------------------------------------------------------------------

@dataclass
class HostTree:
    desc: L.octa_tree_desc
    first_child: np.ndarray   # int32 [num_nodes]
    node_coord: np.ndarray    # int32 [num_nodes][3]
    map_offset: np.ndarray    # int32 [num_nodes]

    @property
    def num_levels(self):
        return self.desc.num_levels

    @property
    def num_nodes(self):
        return self.desc.num_nodes

    @property
    def num_texels(self):
        return self.desc.num_texels

    @property
    def R(self):
        return [self.desc.R[l] for l in range(self.num_levels)]

    @property
    def level_node_start(self):
        return np.array([self.desc.level_node_start[l] for l in range(self.num_levels + 1)])

    @property
    def level_texel_base(self):
        return np.array([self.desc.level_texel_base[l] for l in range(self.num_levels + 1)])


def _two_call(fn, *head):
    desc = L.octa_tree_desc()
    L.check(fn(*head, C.byref(desc), None, None, None), fn.__name__)
    n = desc.num_nodes
    fc = np.empty(n, np.int32)
    nc = np.empty((n, 3), np.int32)
    mo = np.empty(n, np.int32)
    L.check(fn(*head, C.byref(desc), fc.ctypes.data_as(C.c_void_p), nc.ctypes.data_as(C.c_void_p),
               mo.ctypes.data_as(C.c_void_p)), fn.__name__)
    return HostTree(desc, fc, nc, mo)


def octree_build(seed, max_depth, p_base, R):
    Ra = np.ascontiguousarray(R, dtype=np.int32)
    assert len(Ra) == max_depth + 1
    return _two_call(_lib().octree_build, C.c_uint64(seed), C.c_int32(max_depth),
                     C.c_double(p_base), Ra.ctypes.data_as(C.c_void_p))


def octree_from_flags(flags, max_depth, R):
    fl = np.ascontiguousarray(flags, dtype=np.uint8)
    Ra = np.ascontiguousarray(R, dtype=np.int32)
    fp = fl.ctypes.data_as(C.c_void_p) if len(fl) else None
    return _two_call(_lib().octree_from_flags, fp, C.c_int64(len(fl)), C.c_int32(max_depth),
                     Ra.ctypes.data_as(C.c_void_p))


# ---------------------------------------------------------------------------
# scenes and queries (device)
# ---------------------------------------------------------------------------

class Scene:
    """One octree with its feature table and decoder on the device.

    tables: tensor [num_texels][F] float32/float16; weights: list of tensors
    [out][in] (float32 or bfloat16), stored back to back.
    """

    def __init__(self, tree: HostTree, tables, weights, device="cuda",
                 query_form=L.OCTA_FORM_CELL_BILINEAR):
        self.tree = tree
        self.query_form = int(query_form)
        self.device = torch.device(device)
        self.first_child = torch.from_numpy(tree.first_child).to(self.device)
        self.map_offset = torch.from_numpy(tree.map_offset).to(self.device)
        self.tables = tables
        self.widths = [int(weights[0].shape[1])] + [int(W.shape[0]) for W in weights]
        self.weights = torch.cat([W.reshape(-1) for W in weights]).contiguous()
        self.set_tables(tables)

    def set_tables(self, tables):
        assert tables.is_contiguous() and tables.shape[0] == self.tree.num_texels
        self.tables = tables

    def set_weights_flat(self, flat):
        assert flat.numel() == self.weights.numel()
        self.weights = flat

    @property
    def F(self):
        return int(self.tables.shape[1])

    def weight_slices(self):
        out, off = [], 0
        for a, b in zip(self.widths[:-1], self.widths[1:]):
            out.append((off, b, a))
            off += a * b
        return out

    def as_c(self):
        s = L.octa_scene()
        s.first_child = self.first_child.data_ptr()
        s.map_offset = self.map_offset.data_ptr()
        s.tables = self.tables.data_ptr()
        s.weights = self.weights.data_ptr()
        s.num_levels = self.tree.num_levels
        s.num_nodes = self.tree.num_nodes
        s.num_texels = self.tree.num_texels
        for l, r in enumerate(self.tree.R):
            s.R[l] = r
        s.F = self.F
        s.table_dtype = _DT[self.tables.dtype]
        s.weight_dtype = _DT[self.weights.dtype]
        s.n_layers = len(self.widths) - 1
        for i, w in enumerate(self.widths):
            s.widths[i] = w
        s.query_form = self.query_form
        return s


def _scene_array(scenes):
    if isinstance(scenes, Scene):
        scenes = [scenes]
    arr = (L.octa_scene * len(scenes))(*[s.as_c() for s in scenes])
    return arr, len(scenes)


def _queries(x, omega, counts):
    q = L.octa_queries()
    n = int(x.shape[0])
    q.x = x.data_ptr() if n else None
    q.omega = omega.data_ptr() if n else None
    q.n = n
    counts = [n] if counts is None else list(counts)
    assert sum(counts) == n
    acc = 0
    q.scene_start[0] = 0
    for i, c in enumerate(counts):
        acc += c
        q.scene_start[i + 1] = acc
    return q


def octa_encode(scenes, x, omega, counts=None, feat_dtype=torch.float32, want_nodes=False,
                want_addr=False, status=None, stream=None, normal=None, disparity=None):
    """The encoding alone (features [n][W]); normal [n][3] and disparity [n]
    are the shifted form's inputs."""
    arr, ns = _scene_array(scenes)
    sl = [scenes] if isinstance(scenes, Scene) else scenes
    kmax = max(s.tree.num_levels for s in sl)
    W = max(s.tree.num_levels * s.F for s in sl)
    n = x.shape[0]
    dev = x.device
    feat = torch.zeros((n, W), dtype=feat_dtype, device=dev)
    nodes = torch.empty((n, kmax), dtype=torch.int32, device=dev) if want_nodes else None
    per_level = 4 if sl[0].query_form == L.OCTA_FORM_CELL_BILINEAR else 24
    addr = torch.empty((n, kmax, per_level), dtype=torch.int32, device=dev) if want_addr else None
    q = _queries(x, omega, counts)
    q.normal = normal.data_ptr() if normal is not None and n else None
    q.disparity = disparity.data_ptr() if disparity is not None and n else None
    L.check(_lib().octa_encode(arr, ns, C.byref(q), _ptr(feat), _DT[feat_dtype], W, _ptr(nodes),
                               _ptr(addr), _ptr(status), _stream(stream)), "octa_encode")
    return feat, nodes, addr


def _set_extras(q, n, normal=None, disparity=None, attrs=None):
    """The shifted form's normal / disparity and Eq. 12's attributes."""
    q.normal = normal.data_ptr() if normal is not None and n else None
    q.disparity = disparity.data_ptr() if disparity is not None and n else None
    if attrs is not None:
        q.attrs = attrs.data_ptr() if n else None
        q.n_attrs = int(attrs.shape[1])


def octa_query_fwd(scenes, x, omega, counts=None, want_nodes=False, want_addr=False, rgb=None,
                   status=None, stream=None, normal=None, disparity=None, attrs=None):
    arr, ns = _scene_array(scenes)
    sl = [scenes] if isinstance(scenes, Scene) else scenes
    kmax = max(s.tree.num_levels for s in sl)
    n = x.shape[0]
    dev = x.device
    if rgb is None:
        rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
    nodes = torch.empty((n, kmax), dtype=torch.int32, device=dev) if want_nodes else None
    per_level = 4 if sl[0].query_form == L.OCTA_FORM_CELL_BILINEAR else 24
    addr = torch.empty((n, kmax, per_level), dtype=torch.int32, device=dev) if want_addr else None
    q = _queries(x, omega, counts)
    _set_extras(q, n, normal, disparity, attrs)
    L.check(_lib().octa_query_fwd(arr, ns, C.byref(q), _ptr(rgb), _ptr(nodes), _ptr(addr),
                                  _ptr(status), _stream(stream)), "octa_query_fwd")
    return rgb, nodes, addr


def octa_query_bwd(scenes, x, omega, d_rgb, grads, counts=None, status=None, stream=None,
                   attrs=None, normal=None, disparity=None, d_disparity=None):
    """grads: list of (d_tables fp32, d_weights fp32) per scene; accumulated.
    d_disparity [n] (shifted form, optional) receives dL/dd per query."""
    arr, ns = _scene_array(scenes)
    g = (L.octa_scene_grads * ns)(*[L.octa_scene_grads(dt.data_ptr(), dw.data_ptr())
                                    for dt, dw in grads])
    n = int(x.shape[0])
    q = _queries(x, omega, counts)
    _set_extras(q, n, normal, disparity, attrs)
    q.d_disparity = d_disparity.data_ptr() if d_disparity is not None and n else None
    L.check(_lib().octa_query_bwd(arr, ns, C.byref(q), _ptr(d_rgb), g, _ptr(status),
                                  _stream(stream)), "octa_query_bwd")


def _set_norm(pr, norm_pairs):
    if norm_pairs is not None:
        for i, m in enumerate(norm_pairs):
            pr.norm_pairs[i] = int(m)


def _set_shift(pr, n, shift):
    """The shifted form's pair inputs and outputs: shift = (normal, normal2,
    disparity, disparity2, d_disparity or None, d_disparity2 or None)."""
    if shift is None:
        return
    names = ("normal", "normal2", "disparity", "disparity2", "d_disparity", "d_disparity2")
    for nm, t in zip(names, shift):
        setattr(pr, nm, t.data_ptr() if t is not None and n else None)


def octa_train_fused(scenes, x, omega, x2, omega2, E, w, grads, loss_out, counts=None, eps=1e-2,
                     rhs_grad=True, scaler=None, status=None, stream=None, norm_pairs=None,
                     shift=None):
    """Fused forward + Eq. 14 loss + backward over training pairs (BF16
    decoders on the tensor cores, FP32 decoders on the FP32 engine); shift:
    the shifted form's tensors (_set_shift)."""
    arr, ns = _scene_array(scenes)
    g = (L.octa_scene_grads * ns)(*[L.octa_scene_grads(dt.data_ptr(), dw.data_ptr())
                                    for dt, dw in grads])
    pr = L.octa_pairs()
    n = int(x.shape[0])
    pr.x, pr.omega, pr.x2, pr.omega2 = (t.data_ptr() if n else None for t in (x, omega, x2, omega2))
    pr.E, pr.w = (t.data_ptr() if n else None for t in (E, w))
    pr.n = n
    counts = [n] if counts is None else list(counts)
    acc = 0
    for i, c in enumerate(counts):
        acc += c
        pr.scene_start[i + 1] = acc
    _set_norm(pr, norm_pairs)
    _set_shift(pr, n, shift)
    L.check(_lib().octa_train_fused(arr, ns, C.byref(pr), C.c_float(eps), int(bool(rhs_grad)),
                                    _ptr(scaler), _ptr(loss_out), g, _ptr(status), _stream(stream)),
            "octa_train_fused")


def octa_train_step_batched(scenes, x, omega, x2, omega2, E, w, grads, groups, loss_out, scaler, ws,
                            counts=None, eps=1e-2, rhs_grad=True, beta1=0.9, beta2=0.999,
                            adam_eps=1e-8, timeout_ns=0, extra_arrivals=0, status=None,
                            stream=None, norm_pairs=None, skip_first_mma=0):
    """Whole training step (fused pass + Adam) in one persistent launch."""
    arr, ns = _scene_array(scenes)
    g = (L.octa_scene_grads * ns)(*[L.octa_scene_grads(dt.data_ptr(), dw.data_ptr())
                                    for dt, dw in grads])
    pg = (L.octa_param_group * len(groups))(*[gr.as_c() for gr in groups])
    pr = L.octa_pairs()
    n = int(x.shape[0])
    pr.x, pr.omega, pr.x2, pr.omega2 = (t.data_ptr() for t in (x, omega, x2, omega2))
    pr.E, pr.w = E.data_ptr(), w.data_ptr()
    pr.n = n
    counts = [n] if counts is None else list(counts)
    acc = 0
    for i, c in enumerate(counts):
        acc += c
        pr.scene_start[i + 1] = acc
    _set_norm(pr, norm_pairs)
    opt = L.octa_step_options(timeout_ns, extra_arrivals, int(skip_first_mma))
    cfg = L.octa_adam_cfg(beta1, beta2, adam_eps)
    L.check(_lib().octa_train_step_batched(arr, ns, C.byref(pr), g, pg, len(groups), C.c_float(eps),
                                           int(bool(rhs_grad)), C.byref(cfg), _ptr(scaler),
                                           _ptr(loss_out), C.byref(opt), _ptr(ws), ws.numel(),
                                           _ptr(status), _stream(stream)),
            "octa_train_step_batched")


# ---------------------------------------------------------------------------
# loss, optimiser
# ---------------------------------------------------------------------------

SCALER_BYTES = C.sizeof(L.octa_scaler)


def make_scaler(scale=2.0 ** 15, growth_interval=2000, device="cuda"):
    s = L.octa_scaler()
    s.scale = scale
    s.inv_scale_used = 1.0 / scale
    s.growth_interval = growth_interval
    raw = bytes(s)
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)


def read_scaler(buf):
    raw = bytes(buf.cpu().numpy().tobytes())
    return L.octa_scaler.from_buffer_copy(raw)


def workspace(op, n, device="cuda"):
    nbytes = _lib().octa_workspace_bytes(op, n)
    return torch.zeros(nbytes, dtype=torch.uint8, device=device)


def residual_loss(Lp, Ls, E, w, dLp, dLs, loss_out, ws, eps=1e-2, rhs_grad=True, scaler=None,
                  stream=None):
    n = int(Lp.shape[0])
    L.check(_lib().residual_loss(_ptr(Lp), _ptr(Ls), _ptr(E), _ptr(w), n, C.c_float(eps),
                                 int(bool(rhs_grad)), _ptr(scaler), _ptr(loss_out), _ptr(dLp),
                                 _ptr(dLs), _ptr(ws), ws.numel(), _stream(stream)),
            "residual_loss")


def residual_loss_multi(Lp, Ls, E, w, dLp, dLs, loss_out, ws, eps=1e-2, rhs_grad=True,
                        scaler=None, stream=None):
    """Eq. 14 against Eq. 3's M-sample target: Lp, E, dLp [N][3]; Ls, w, dLs
    [N][M][3] (dLs may be None without rhs_grad)."""
    n, M = int(w.shape[0]), int(w.shape[1])
    L.check(_lib().residual_loss_multi(_ptr(Lp), _ptr(Ls), _ptr(E), _ptr(w), n, M, C.c_float(eps),
                                       int(bool(rhs_grad)), _ptr(scaler), _ptr(loss_out),
                                       _ptr(dLp), _ptr(dLs), _ptr(ws), ws.numel(),
                                       _stream(stream)),
            "residual_loss_multi")


class Prims:
    """The synthetic scene on the device for octa_trace_rays: planes [P][13]
    and spheres [S][4] float32 (see inputs.scene_arrays)."""

    def __init__(self, planes, spheres, device="cuda"):
        dev = torch.device(device)
        self.planes = torch.as_tensor(planes, dtype=torch.float32).reshape(-1, 13).to(dev).contiguous()
        self.spheres = torch.as_tensor(spheres, dtype=torch.float32).reshape(-1, 4).to(dev).contiguous()

    def as_c(self):
        p = L.octa_prims()
        p.planes = self.planes.data_ptr() if self.planes.numel() else None
        p.spheres = self.spheres.data_ptr() if self.spheres.numel() else None
        p.n_planes = int(self.planes.shape[0])
        p.n_spheres = int(self.spheres.shape[0])
        return p


def octa_trace_rays(prims, origin, direction, rays_per_origin=1, t_min=1e-4, hit=None,
                    query_dir=None, want_prim=False, want_t=False, stream=None):
    """x'(omega_i) of Eq. 2 for every ray (origin[i // rays_per_origin],
    direction[i]); returns (hit, query_dir, prim, t), the last three None
    unless asked for (query_dir: pass a buffer or True)."""
    n = int(direction.shape[0])
    dev = direction.device
    if hit is None:
        hit = torch.empty((n, 3), dtype=torch.float32, device=dev)
    if query_dir is True:
        query_dir = torch.empty((n, 3), dtype=torch.float32, device=dev)
    prim = torch.empty(n, dtype=torch.int32, device=dev) if want_prim else None
    t = torch.empty(n, dtype=torch.float32, device=dev) if want_t else None
    pc = prims.as_c()
    L.check(_lib().octa_trace_rays(C.byref(pc), _ptr(origin), int(rays_per_origin),
                                   _ptr(direction), n, C.c_float(t_min), _ptr(hit),
                                   _ptr(query_dir), _ptr(prim), _ptr(t), _stream(stream)),
            "octa_trace_rays")
    return hit, query_dir, prim, t


class Predictor:
    """The disparity predictor g_psi on the device: hash tables [L][T][2]
    float32 (T a power of two), per-level resolutions, and the MLP
    W1 [64][2L+3], W2 [64][64], W3 [1][64] float32."""

    def __init__(self, table, res, weights, device="cuda", tensor_cores=False):
        dev = torch.device(device)
        self.table = torch.as_tensor(table, dtype=torch.float32).to(dev).contiguous()
        L_, T, F = self.table.shape
        assert F == 2 and T & (T - 1) == 0 and len(res) == L_
        self.res = [int(r) for r in res]
        self.weights = torch.cat([torch.as_tensor(W, dtype=torch.float32).reshape(-1)
                                  for W in weights]).to(dev).contiguous()
        # tensor_cores: the MLP in BF16 on the tcgen05 path
        self.weights_bf16 = self.weights.to(torch.bfloat16).contiguous() if tensor_cores else None

    def as_c(self):
        p = L.octa_predictor()
        p.table = self.table.data_ptr()
        p.weights = self.weights.data_ptr()
        p.weights_bf16 = self.weights_bf16.data_ptr() if self.weights_bf16 is not None else None
        p.levels = len(self.res)
        p.log2_T = int(self.table.shape[1]).bit_length() - 1
        for i, r in enumerate(self.res):
            p.res[i] = r
        return p


def octa_disparity(pred, x, omega, normal, out=None, stream=None):
    """d = g_psi(x, omega_r) per query (Eq. 7)."""
    n = int(x.shape[0])
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=x.device)
    q = _queries(x, omega, None)
    q.normal = normal.data_ptr() if n else None
    pc = pred.as_c()
    L.check(_lib().octa_disparity(C.byref(pc), C.byref(q), _ptr(out), _stream(stream)),
            "octa_disparity")
    return out


def octa_disparity_bwd(pred, x, omega, normal, d_disp, d_table, d_weights, stream=None):
    """g_psi's backward: accumulates the gradients of sum_q d_disp[q] d_q into
    d_table (layout of pred.table) and d_weights (layout of pred.weights)."""
    n = int(x.shape[0])
    q = _queries(x, omega, None)
    q.normal = normal.data_ptr() if n else None
    pc = pred.as_c()
    L.check(_lib().octa_disparity_bwd(C.byref(pc), C.byref(q), _ptr(d_disp), _ptr(d_table),
                                      _ptr(d_weights), _stream(stream)), "octa_disparity_bwd")


@dataclass
class ParamGroup:
    param: torch.Tensor
    grad: torch.Tensor
    m: torch.Tensor
    v: torch.Tensor
    lr: float
    work: torch.Tensor | None = None

    def as_c(self):
        g = L.octa_param_group()
        g.param = self.param.data_ptr()
        g.grad = self.grad.data_ptr()
        g.m = self.m.data_ptr()
        g.v = self.v.data_ptr()
        g.work = self.work.data_ptr() if self.work is not None else None
        g.work_dtype = _DT[self.work.dtype] if self.work is not None else L.OCTA_F16
        g.lr = self.lr
        g.n = self.param.numel()
        return g


def adam_step(groups, scaler, ws, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    arr = (L.octa_param_group * len(groups))(*[g.as_c() for g in groups])
    cfg = L.octa_adam_cfg(beta1, beta2, eps)
    L.check(_lib().adam_step(arr, len(groups), C.byref(cfg), _ptr(scaler), _ptr(ws), ws.numel(),
                             _stream(stream)), "adam_step")


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------

class OctaQueryFunction(torch.autograd.Function):
    """L_hat(x, omega) differentiable w.r.t. the feature table and the flat
    decoder weights; backward runs octa_query_bwd (forward recomputed)."""

    @staticmethod
    def forward(ctx, x, omega, tables, weights_flat, scene):
        scene.set_tables(tables.detach())
        scene.set_weights_flat(weights_flat.detach())
        rgb, _, _ = octa_query_fwd(scene, x, omega)
        ctx.save_for_backward(x, omega)
        ctx.scene = scene
        return rgb

    @staticmethod
    def backward(ctx, d_rgb):
        x, omega = ctx.saved_tensors
        sc = ctx.scene
        dT = torch.zeros(sc.tables.shape, dtype=torch.float32, device=x.device)
        dW = torch.zeros(sc.weights.shape, dtype=torch.float32, device=x.device)
        octa_query_bwd(sc, x, omega, d_rgb.contiguous().float(), [(dT, dW)])
        return None, None, dT, dW, None


def octa_query(scene, x, omega, tables, weights_flat):
    return OctaQueryFunction.apply(x, omega, tables, weights_flat, scene)
