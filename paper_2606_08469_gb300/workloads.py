"""Assemble the synthetic workloads (seeded inputs + octree + parameters) on
the device, for tests, the benchmark and the smoke check."""
from __future__ import annotations

import numpy as np
import torch

from . import api
from . import inputs as I
from .train import MultiSampleStep, PredictorState, SceneState, ShiftedTrainStep, TrainStep

_TORCH_DT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}


def table_dtype(cfg):
    return _TORCH_DT[cfg.table_dtype]


def weight_dtype(cfg):
    return _TORCH_DT[cfg.weight_dtype]


def host_params(cfg, tree_seed=None, tables_seed=None, mlp_seed=None, vertex_maps=False):
    """Host tree (library builder) plus FP32 master tables and weights.
    vertex_maps: maps of side R + 1 (vertices of an R-cell grid, for the
    trilinear vertex query form) in place of R x R texel maps."""
    R = [r + 1 for r in cfg.R] if vertex_maps else cfg.R
    tree = api.octree_build(cfg.seed("tree") if tree_seed is None else tree_seed, cfg.max_depth,
                            cfg.p_base, R)
    tables = I.make_tables(cfg.seed("tables") if tables_seed is None else tables_seed,
                           tree.num_texels, cfg.F, cfg.sigma)
    widths = [tree.num_levels * cfg.F] + list(cfg.widths[1:])
    weights = I.make_mlp(cfg.seed("mlp") if mlp_seed is None else mlp_seed, widths)
    return tree, tables, weights


def pairs_on_device(pairs, device="cuda"):
    return {k: torch.from_numpy(getattr(pairs, k)).to(device)
            for k in ("x", "omega", "x2", "omega2", "E", "w")}


def train_step_for(cfg, n_pairs=None, device="cuda", precision=None, query_form=None, **kw):
    """TrainStep of a 'pairs' workload.  precision='f32' forces the FP32 path
    on the same shapes (FP32 tables and weights); query_form='full' queries
    the trilinear vertex form on vertex maps of side R + 1."""
    full = query_form == "full"
    tree, tables, weights = host_params(cfg, vertex_maps=full)
    tdt, wdt = table_dtype(cfg), weight_dtype(cfg)
    if precision == "f32":
        tdt = wdt = torch.float32
    st = SceneState(tree, tables, weights, tdt, wdt, device,
                    query_form=api.L.OCTA_FORM_TRILINEAR_VERTEX if full else
                    api.L.OCTA_FORM_CELL_BILINEAR)
    n = cfg.n if n_pairs is None else n_pairs
    pairs = I.training_pairs(cfg.seed("queries"), n)
    return TrainStep([st], [pairs_on_device(pairs, device)], **kw), (tree, tables, weights, pairs)


def data_parallel_train_step(cfg, rank, world, n_pairs=None, device="cuda", precision=None, **kw):
    """Fused TrainStep of a data-parallel rank: the batch's seeded pairs,
    this rank's contiguous shard, the loss normalised by the whole batch."""
    from .dataparallel import shard_range
    tree, tables, weights = host_params(cfg)
    tdt, wdt = table_dtype(cfg), weight_dtype(cfg)
    if precision == "f32":
        tdt = wdt = torch.float32
    st = SceneState(tree, tables, weights, tdt, wdt, device)
    n = cfg.n if n_pairs is None else n_pairs
    pairs = I.training_pairs(cfg.seed("queries"), n)
    b, e = shard_range(n, rank, world)
    shard = {k: torch.from_numpy(np.ascontiguousarray(getattr(pairs, k)[b:e])).to(device)
             for k in ("x", "omega", "x2", "omega2", "E", "w")}
    step = TrainStep([st], [shard], fused=True, norm_pairs=[n], device=device, **kw)
    return step, (tree, tables, weights, pairs, (b, e))


def data_parallel_rank_step(cfg, rank, world, n_per_rank=None, device="cuda", precision=None,
                            **kw):
    """Fused TrainStep of one rank of a weak-scaling data-parallel job: the
    global batch is world x n_per_rank pairs, rank r holding its own
    n_per_rank seeded pairs (seed of the workload's queries + 7919 r), every
    rank's loss normalised by the global batch."""
    tree, tables, weights = host_params(cfg)
    tdt, wdt = table_dtype(cfg), weight_dtype(cfg)
    if precision == "f32":
        tdt = wdt = torch.float32
    st = SceneState(tree, tables, weights, tdt, wdt, device)
    n = cfg.n if n_per_rank is None else n_per_rank
    pairs = I.training_pairs(cfg.seed("queries") + 7919 * rank, n)
    step = TrainStep([st], [pairs_on_device(pairs, device)], fused=True, norm_pairs=[n * world],
                     device=device, **kw)
    return step, (tree, tables, weights, pairs)


def batched_train_step(device="cuda", counts=None, precision=None, **kw):
    """TrainStep of the batched workload (8 scenes); counts overrides the
    per-scene pair counts."""
    cfg = I.WORKLOADS["batched"]
    counts = I.batched_pair_counts(cfg) if counts is None else counts
    states, plist, host = [], [], []
    for s, n in enumerate(counts):
        sc = I.batched_scene_config(s, cfg)
        tree = api.octree_build(I.batched_seed(s, "tree"), sc.max_depth, sc.p_base, sc.R)
        tables = I.make_tables(I.batched_seed(s, "tables"), tree.num_texels, sc.F, sc.sigma)
        weights = I.make_mlp(I.batched_seed(s, "mlp"), [tree.num_levels * sc.F, 64, 64, 3])
        tdt, wdt = table_dtype(sc), weight_dtype(sc)
        if precision == "f32":
            tdt = wdt = torch.float32
        states.append(SceneState(tree, tables, weights, tdt, wdt, device))
        pairs = I.training_pairs(I.batched_seed(s, "queries"), n)
        plist.append(pairs_on_device(pairs, device))
        host.append((tree, tables, weights, pairs))
    return TrainStep(states, plist, **kw), host


def forward_scene(cfg, device="cuda", precision=None):
    """Device scene of a forward workload (tables/weights in the config's
    precision, or FP32 with precision='f32')."""
    tree, tables, weights = host_params(cfg)
    tdt, wdt = table_dtype(cfg), weight_dtype(cfg)
    if precision == "f32":
        tdt = wdt = torch.float32
    T = torch.from_numpy(tables).to(device).to(tdt).contiguous()
    Ws = [torch.from_numpy(W).to(device).to(wdt) for W in weights]
    return api.Scene(tree, T, Ws, device=device), (tree, tables, weights)


def queries_for(cfg, n=None):
    """Host (x, omega) of a forward workload."""
    if cfg.kind == "uniform":
        return I.uniform_queries(cfg.seed("queries"), cfg.n if n is None else n)
    if cfg.kind == "gbuffer":
        w, h = cfg.extra["width"], cfg.extra["height"]
        return I.gbuffer_queries(cfg.seed("queries"), w, h)
    pairs = I.training_pairs(cfg.seed("queries"), cfg.n if n is None else n)
    return pairs.x, pairs.omega


def to_dev(a, device="cuda"):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


def multi_sample_step_for(cfg, n, M, device="cuda", precision=None, seed=None, **kw):
    """MultiSampleStep of a 'pairs' workload's scene parameters on n LHS
    samples with M RHS samples each (training_samples batch; secondary hits
    ray cast on the device every step)."""
    tree, tables, weights = host_params(cfg)
    tdt, wdt = table_dtype(cfg), weight_dtype(cfg)
    if precision == "f32":
        tdt = wdt = torch.float32
    st = SceneState(tree, tables, weights, tdt, wdt, device)
    smp = I.training_samples(cfg.seed("queries") if seed is None else seed, n, M)
    dev = torch.device(device)
    arrays = {k: torch.from_numpy(getattr(smp, k)).to(dev) for k in ("x", "omega", "E", "omega_i", "w")}
    prims = api.Prims(smp.planes, smp.spheres, device=dev)
    return MultiSampleStep(st, prims, arrays, device=device, **kw), (tree, tables, weights, smp)


# the disparity predictor of the shifted-form workloads: 8 hash levels of
# 2^16 entries, resolutions 16 ... 512 on a geometric progression
PREDICTOR_LEVELS = 8
PREDICTOR_LOG2_T = 16
PREDICTOR_RES = [int(np.floor(16 * (512 / 16) ** (l / 7))) for l in range(PREDICTOR_LEVELS)]


def shifted_train_step_for(cfg, n_pairs=None, device="cuda", precision=None, attrs=0, **kw):
    """ShiftedTrainStep of a 'pairs' workload: the paper's full model on the
    workload's tree with vertex maps of side R + 1 (the shifted form), the
    workload's table and decoder precisions (precision='f32': FP32), and
    the predictor above (FP32 MLP; on the tensor cores when the decoder is
    BF16)."""
    tree, tables, weights = host_params(cfg, vertex_maps=True)
    tdt, wdt = table_dtype(cfg), weight_dtype(cfg)
    if precision == "f32":
        tdt = wdt = torch.float32
    st = SceneState(tree, tables, weights, tdt, wdt, device, query_form=api.L.OCTA_FORM_SHIFTED)
    ptab, pw = I.predictor_params(cfg.seed("mlp") + 7, PREDICTOR_LEVELS, PREDICTOR_LOG2_T)
    ps = PredictorState(ptab, PREDICTOR_RES, pw, device, tensor_cores=wdt == torch.bfloat16)
    n = cfg.n if n_pairs is None else n_pairs
    pairs, n1, n2 = I.training_pairs_with_normals(cfg.seed("queries"), n)
    arrays = pairs_on_device(pairs, device)
    arrays["normal"] = to_dev(n1, device)
    arrays["normal2"] = to_dev(n2, device)
    return ShiftedTrainStep(st, ps, arrays, device=device, **kw), \
        (tree, tables, weights, (ptab, PREDICTOR_RES, pw), pairs, n1, n2)
