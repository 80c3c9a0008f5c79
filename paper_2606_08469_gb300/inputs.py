"""Seeded synthetic inputs for the OctaOctree query and its training step.

This module only draws random inputs (numpy PCG64); it holds none of the
method's arithmetic (no tree walk, no octahedral encoding, no interpolation,
no network, no loss).  Both the CUDA path and the FP64 oracle are fed from
here, so the two share inputs and nothing else.

The paper's scenes (Section 4.1: Mitsuba 3 renderings of Bathroom,
Cornell-box, Kitchen, Living-room, Veach-ajar, 1024x1024 and 1280x720) are
not available; these generators stand in for them with the same query-set
shapes: surface points on planes and spheres inside the unit cube, directions
on the hemisphere about the normal (training, Section 3.6), and a pinhole
G-buffer with glossy reflection directions (inference, Section 3.6 last
paragraph).

Seeds per configuration index i: tree 1000+i, tables 2000+i, MLP 3000+i,
queries 4000+i.  The batched configuration uses 1400+s, 2400+s, 3400+s,
4400+s for scene s and 4499 for the per-scene query counts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Angular resolution per level for the deeper trees (coarse levels get the
# finer octahedral maps, Section 3.4); depth 9 extends it with R=8.
R_DEEP = [64, 64, 32, 32, 16, 16, 8, 8, 8, 8]


@dataclass
class Config:
    """One workload: tree shape, table format, MLP widths and batch size."""
    index: int
    max_depth: int
    p_base: float
    R: list
    F: int
    table_dtype: str          # "f32" or "f16"
    sigma: float              # std of the initial features
    widths: list              # MLP widths, widths[0] = K*F, last = 3
    weight_dtype: str         # "f32" or "bf16"
    n: int                    # queries (forward configs) or pairs (training)
    kind: str                 # "uniform" | "pairs" | "gbuffer" | "batched"
    loss_scaling: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def num_levels(self):
        return self.max_depth + 1

    def seed(self, what):
        base = {"tree": 1000, "tables": 2000, "mlp": 3000, "queries": 4000}[what]
        return base + self.index


# The workloads by name (their index only seeds the generators):
# forward_small  16,384 uniform queries on a depth-4 tree, FP32 decoder 20-32-32-3
# train_f32      262,144 training pairs on a depth-6 tree, FP32 decoder 56-64-64-3
# train_bf16     1,048,576 pairs on a depth-8 tree, FP16 tables, BF16 72-64-64-64-3
# gbuffer_frame  a 1280x720 G-buffer frame on a depth-8 tree, BF16 72-64-64-3
# batched        eight scenes of depth 4..9, log-uniform pair counts, BF16 80-64-64-3
WORKLOADS = {
    "forward_small": Config(0, 4, 0.6, [16, 16, 8, 8, 8], 4, "f32", 0.1, [20, 32, 32, 3], "f32",
              16384, "uniform"),
    "train_f32": Config(1, 6, 0.6, [32, 32, 16, 16, 8, 8, 8], 8, "f32", 0.01, [56, 64, 64, 3], "f32",
              262144, "pairs"),
    "train_bf16": Config(2, 8, 0.6, R_DEEP[:9], 8, "f16", 0.01, [72, 64, 64, 64, 3], "bf16",
              1048576, "pairs", loss_scaling=True),
    "gbuffer_frame": Config(3, 8, 0.6, R_DEEP[:9], 8, "f16", 0.01, [72, 64, 64, 3], "bf16",
              1280 * 720, "gbuffer", extra={"width": 1280, "height": 720}),
    "batched": Config(4, 9, 0.6, R_DEEP, 8, "f16", 0.01, [80, 64, 64, 3], "bf16",
              0, "batched", loss_scaling=True,
              extra={"depths": [4, 5, 6, 7, 8, 8, 9, 9], "log2_min": 16, "log2_max": 21}),
}


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------

def make_tables(seed, num_texels, F, sigma):
    """Feature tables [num_texels][F] float32 drawn from N(0, sigma^2)."""
    return rng(seed).normal(0.0, sigma, size=(int(num_texels), F)).astype(np.float32)


def make_mlp(seed, widths):
    """Xavier-uniform weight matrices W_i [widths[i+1]][widths[i]] (float32).

    No biases (the decoder is bias-free, as tiny-cuda-nn's fused MLPs are).
    """
    g = rng(seed)
    mats = []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        a = math.sqrt(6.0 / (fan_in + fan_out))
        mats.append(g.uniform(-a, a, size=(fan_out, fan_in)).astype(np.float32))
    return mats


# ---------------------------------------------------------------------------
# directions and points
# ---------------------------------------------------------------------------

def _unit_vectors(g, n):
    """Uniform directions on S^2 (normalised Gaussians), float64."""
    v = g.normal(size=(n, 3))
    nrm = np.linalg.norm(v, axis=1)
    bad = nrm < 1e-12
    while bad.any():
        v[bad] = g.normal(size=(int(bad.sum()), 3))
        nrm = np.linalg.norm(v, axis=1)
        bad = nrm < 1e-12
    return v / nrm[:, None]


def uniform_queries(seed, n):
    """x ~ U[0,1)^3 and omega uniform on the sphere (float32 [n][3] each)."""
    g = rng(seed)
    x = g.random((n, 3)).astype(np.float32)
    w = _unit_vectors(g, n).astype(np.float32)
    return x, w


def _tangent_frame(nrm):
    a = np.where(np.abs(nrm[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    t1 = np.cross(nrm, a)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(nrm, t1)
    return t1, t2


@dataclass
class Primitives:
    """Planes (point p, normal n, optional half-size) and spheres (c, r)."""
    plane_p: np.ndarray
    plane_n: np.ndarray
    plane_half: np.ndarray     # inf for unbounded training planes
    sphere_c: np.ndarray
    sphere_r: np.ndarray
    alpha: np.ndarray          # roughness per primitive (planes first, then spheres)


def make_primitives(g, n_planes, n_spheres, patch=False):
    plane_n = _unit_vectors(g, n_planes)
    plane_p = g.uniform(0.2, 0.8, size=(n_planes, 3))
    if patch:
        plane_half = g.uniform(0.05, 0.25, size=n_planes)
    else:
        plane_half = np.full(n_planes, np.inf)
    sphere_c = g.uniform(0.2, 0.8, size=(n_spheres, 3))
    sphere_r = g.uniform(0.05, 0.2, size=n_spheres)
    alpha = g.uniform(0.05, 0.6, size=n_planes + n_spheres)
    return Primitives(plane_p, plane_n, plane_half, sphere_c, sphere_r, alpha)


def sample_surface_points(g, prims, n):
    """Points (and normals) on a uniformly chosen primitive, inside [0,1]^3."""
    n_pl = len(prims.plane_p)
    n_sp = len(prims.sphere_c)
    which = g.integers(0, n_pl + n_sp, size=n)
    x = np.empty((n, 3))
    nrm = np.empty((n, 3))
    for k in range(n_pl + n_sp):
        idx = np.nonzero(which == k)[0]
        m = len(idx)
        if m == 0:
            continue
        got_x = np.empty((0, 3))
        got_n = np.empty((0, 3))
        while len(got_x) < m:
            need = m - len(got_x)
            draw = max(64, 4 * need)
            if k < n_pl:
                p0 = prims.plane_p[k]
                nn = prims.plane_n[k][None, :]
                t1, t2 = _tangent_frame(nn)
                ab = g.uniform(-1.4, 1.4, size=(draw, 2))
                pts = p0 + ab[:, :1] * t1 + ab[:, 1:] * t2
                nrms = np.repeat(nn, draw, axis=0)
            else:
                s = k - n_pl
                u = _unit_vectors(g, draw)
                pts = prims.sphere_c[s] + prims.sphere_r[s] * u
                nrms = u
            ok = np.all((pts >= 0.0) & (pts <= 1.0), axis=1)
            got_x = np.concatenate([got_x, pts[ok]])[:m]
            got_n = np.concatenate([got_n, nrms[ok]])[:m]
        x[idx] = got_x
        nrm[idx] = got_n
    return x, nrm


def unit_vectors(g, n):
    """Uniform directions on S^2 (float64 [n][3])."""
    return _unit_vectors(g, n)


def scene_arrays(prims):
    """The scene as the ray caster takes it: planes [P][13] float32 (point,
    unit normal, the two tangents of the patch frame, half-size; inf for an
    unbounded plane) and spheres [S][4] float32 (centre, radius)."""
    t1, t2 = _tangent_frame(prims.plane_n)
    planes = np.concatenate([prims.plane_p, prims.plane_n, t1, t2, prims.plane_half[:, None]],
                            axis=1).astype(np.float32)
    spheres = np.concatenate([prims.sphere_c, prims.sphere_r[:, None]], axis=1).astype(np.float32)
    return np.ascontiguousarray(planes), np.ascontiguousarray(spheres)


def hemisphere_directions(g, nrm):
    """Uniform directions on the hemisphere about each normal."""
    w = _unit_vectors(g, len(nrm))
    flip = np.sum(w * nrm, axis=1) < 0
    w[flip] *= -1.0
    return w


@dataclass
class TrainingPairs:
    """One LHS query (x, omega) per pair and one RHS sample (x', omega')."""
    x: np.ndarray        # [n][3] float32, primary position
    omega: np.ndarray    # [n][3] float32, primary outgoing direction
    x2: np.ndarray       # [n][3] float32, secondary hit position x'
    omega2: np.ndarray   # [n][3] float32, sampled incident direction omega'
    E: np.ndarray        # [n][3] float32, emitted radiance
    w: np.ndarray        # [n][3] float32, f_r |n.omega'| / p(omega') weight

    @property
    def n(self):
        return len(self.x)


def training_pairs(seed, n, n_planes=8, n_spheres=8):
    """Training batch: 16 planes/spheres in the unit cube, omega on the
    hemisphere about the normal, omega' uniform, 5% emissive points and a
    U[0,1]^3 BSDF*cos/pdf weight."""
    return training_pairs_with_normals(seed, n, n_planes, n_spheres)[0]


def training_pairs_with_normals(seed, n, n_planes=8, n_spheres=8):
    """training_pairs (the same draws, so the same pairs) and the surface
    normals at x and at x' (float32 [n][3] each), which the disparity-
    shifted lookup reflects its query directions about."""
    g = rng(seed)
    prims = make_primitives(g, n_planes, n_spheres)
    x, nrm = sample_surface_points(g, prims, n)
    om = hemisphere_directions(g, nrm)
    x2, nrm2 = sample_surface_points(g, prims, n)
    om2 = _unit_vectors(g, n)
    emissive = g.random(n) < 0.05
    E = g.random((n, 3)) * emissive[:, None]
    w = g.random((n, 3))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return TrainingPairs(f32(x), f32(om), f32(x2), f32(om2), f32(E), f32(w)), f32(nrm), f32(nrm2)


def predictor_params(seed, levels=8, log2_T=16, table_scale=1e-1):
    """Parameters of the disparity predictor g_psi: hash tables
    [levels][2^log2_T][2] uniform in [-table_scale, table_scale] and
    Xavier-uniform weights of the bias-free MLP (2 levels + 3) -> 64 -> 64
    -> 1.  The per-level grid resolutions are the caller's."""
    g = rng(seed)
    table = g.uniform(-table_scale, table_scale, (levels, 1 << log2_T, 2)).astype(np.float32)
    return table, make_mlp(seed + 1, [2 * levels + 3, 64, 64, 1])


@dataclass
class TrainingSamples:
    """LHS samples with M sampled incident directions each (Eq. 3); the
    secondary positions x'^m come from ray casting the scene (Eq. 2)."""
    x: np.ndarray        # [n][3] float32, LHS position on a primitive
    omega: np.ndarray    # [n][3] float32, outgoing direction
    E: np.ndarray        # [n][3] float32, emitted radiance
    omega_i: np.ndarray  # [n][M][3] float32, incident directions (hemisphere about the normal)
    w: np.ndarray        # [n][M][3] float32, f_r |n.omega_i| / p(omega_i)
    planes: np.ndarray   # scene_arrays(prims)
    spheres: np.ndarray

    @property
    def n(self):
        return len(self.x)

    @property
    def M(self):
        return self.omega_i.shape[1]


def training_samples(seed, n, M, n_planes=8, n_spheres=8):
    """The training batch of Section 4's regime: n LHS samples as in
    training_pairs (16 unbounded planes and spheres, omega on the hemisphere,
    5% emissive points), each with M incident directions drawn uniformly on
    the hemisphere about the point's normal and U[0,1]^3 weights."""
    g = rng(seed)
    prims = make_primitives(g, n_planes, n_spheres)
    x, nrm = sample_surface_points(g, prims, n)
    om = hemisphere_directions(g, nrm)
    emissive = g.random(n) < 0.05
    E = g.random((n, 3)) * emissive[:, None]
    oi = hemisphere_directions(g, np.repeat(nrm, M, axis=0)).reshape(n, M, 3)
    w = g.random((n, M, 3))
    planes, spheres = scene_arrays(prims)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return TrainingSamples(f32(x), f32(om), f32(E), f32(oi), f32(w), planes, spheres)


# ---------------------------------------------------------------------------
# G-buffer for the real-time inference workload
# ---------------------------------------------------------------------------

def _intersect(o, d, prims):
    """Nearest hit of rays (o, d) with patches, spheres and the 6 box walls."""
    n = len(d)
    best_t = np.full(n, np.inf)
    best_n = np.zeros((n, 3))
    best_a = np.zeros(n)
    eps = 1e-7
    # plane patches
    for k in range(len(prims.plane_p)):
        nn = prims.plane_n[k]
        den = d @ nn
        with np.errstate(divide="ignore", invalid="ignore"):
            t = ((prims.plane_p[k] - o) @ nn) / den
        hit = o + t[:, None] * d
        t1, t2 = _tangent_frame(nn[None, :])
        rel = hit - prims.plane_p[k]
        a = rel @ t1[0]
        b = rel @ t2[0]
        h = prims.plane_half[k]
        ok = (np.abs(den) > 1e-12) & (t > eps) & (np.abs(a) <= h) & (np.abs(b) <= h) & (t < best_t)
        best_t = np.where(ok, t, best_t)
        best_n[ok] = nn
        best_a[ok] = prims.alpha[k]
    # spheres
    n_pl = len(prims.plane_p)
    for s in range(len(prims.sphere_c)):
        oc = o - prims.sphere_c[s]
        bq = np.sum(oc * d, axis=1)
        cq = np.sum(oc * oc, axis=1) - prims.sphere_r[s] ** 2
        disc = bq * bq - cq
        sq = np.sqrt(np.maximum(disc, 0.0))
        t0 = -bq - sq
        t1v = -bq + sq
        t = np.where(t0 > eps, t0, t1v)
        ok = (disc >= 0) & (t > eps) & (t < best_t)
        best_t = np.where(ok, t, best_t)
        hitp = o + t[:, None] * d
        best_n[ok] = ((hitp - prims.sphere_c[s]) / prims.sphere_r[s])[ok]
        best_a[ok] = prims.alpha[n_pl + s]
    # inner walls of the unit box (backstop: every ray hits one)
    for axis in range(3):
        for wall, wn in ((0.0, 1.0), (1.0, -1.0)):
            with np.errstate(divide="ignore", invalid="ignore"):
                t = (wall - o[:, axis]) / d[:, axis]
            ok = (t > eps) & (t < best_t)
            best_t = np.where(ok, t, best_t)
            nv = np.zeros(3)
            nv[axis] = wn
            best_n[ok] = nv
            best_a[ok] = 0.3
    return best_t, best_n, best_a


def gbuffer_queries(seed, width, height, n_planes=16, n_spheres=16, fov_deg=60.0, chunk=1 << 17):
    """Primary-hit queries of a pinhole camera at (0.5, 0.5, 0.98) looking -z.

    omega is the view direction reflected about a Beckmann-sampled microfacet
    normal (tan^2 theta = -alpha^2 ln(1-u1), phi = 2 pi u2); samples that fall
    below the surface are redrawn (8 tries, then the mirror direction).  Pixel
    order (row-major, top row first) is kept.
    """
    g = rng(seed)
    prims = make_primitives(g, n_planes, n_spheres, patch=True)
    eye = np.array([0.5, 0.5, 0.98])
    tan_half = math.tan(math.radians(fov_deg) / 2.0)
    aspect = width / height
    xs_out = np.empty((width * height, 3), dtype=np.float32)
    ws_out = np.empty((width * height, 3), dtype=np.float32)
    total = width * height
    for start in range(0, total, chunk):
        idx = np.arange(start, min(total, start + chunk))
        px = idx % width
        py = idx // width
        ndc_x = (2.0 * (px + 0.5) / width - 1.0) * tan_half * aspect
        ndc_y = (1.0 - 2.0 * (py + 0.5) / height) * tan_half
        d = np.stack([ndc_x, ndc_y, -np.ones_like(ndc_x)], axis=1)
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        o = np.repeat(eye[None, :], len(idx), axis=0)
        t, nrm, alpha = _intersect(o, d, prims)
        nrm = np.where((np.sum(nrm * d, axis=1) > 0)[:, None], -nrm, nrm)
        hit = np.clip(o + t[:, None] * d, 0.0, 1.0)
        v = -d
        t1, t2 = _tangent_frame(nrm)
        omega = np.empty_like(d)
        todo = np.ones(len(idx), dtype=bool)
        for _ in range(8):
            m_idx = np.nonzero(todo)[0]
            if len(m_idx) == 0:
                break
            u1 = g.random(len(m_idx))
            u2 = g.random(len(m_idx))
            a = alpha[m_idx]
            tan2 = -(a * a) * np.log1p(-u1)
            cos_t = 1.0 / np.sqrt(1.0 + tan2)
            sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
            phi = 2.0 * math.pi * u2
            m = (sin_t * np.cos(phi))[:, None] * t1[m_idx] + (sin_t * np.sin(phi))[:, None] * t2[m_idx] \
                + cos_t[:, None] * nrm[m_idx]
            vm = np.sum(v[m_idx] * m, axis=1)
            wr = 2.0 * vm[:, None] * m - v[m_idx]
            ok = np.sum(wr * nrm[m_idx], axis=1) > 0
            omega[m_idx[ok]] = wr[ok]
            todo[m_idx[ok]] = False
        rest = np.nonzero(todo)[0]
        if len(rest):
            vn = np.sum(v[rest] * nrm[rest], axis=1)
            omega[rest] = 2.0 * vn[:, None] * nrm[rest] - v[rest]
        omega /= np.linalg.norm(omega, axis=1, keepdims=True)
        xs_out[idx] = hit
        ws_out[idx] = omega
    return xs_out, ws_out


# ---------------------------------------------------------------------------
# batched workload
# ---------------------------------------------------------------------------

def batched_pair_counts(cfg=WORKLOADS["batched"]):
    """Per-scene pair counts floor(2^U[16,21]) (log-uniform)."""
    g = rng(4499)
    e = g.uniform(cfg.extra["log2_min"], cfg.extra["log2_max"], size=len(cfg.extra["depths"]))
    return [int(math.floor(2.0 ** v)) for v in e]


def batched_scene_config(s, cfg=WORKLOADS["batched"]):
    """Per-scene configuration of the batched workload (scene s)."""
    depth = cfg.extra["depths"][s]
    K = depth + 1
    return Config(400 + s, depth, cfg.p_base, R_DEEP[:K], cfg.F, cfg.table_dtype, cfg.sigma,
                  [cfg.F * K, 64, 64, 3], cfg.weight_dtype, 0, "pairs", loss_scaling=True)


def batched_seed(s, what):
    return {"tree": 1400, "tables": 2400, "mlp": 3400, "queries": 4400}[what] + s
