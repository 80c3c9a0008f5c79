"""Plain FP64 CPU oracle of the OctaOctree query and its training step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call
this module: only tests, the smoke check and the benchmark's CPU-baseline leg
do.  It shares no code with the CUDA library (no kernels, headers, helpers or
table generators); both sides receive the same seeded inputs and nothing else.

Every function follows the paper's definitions step by step, in FP64, with
numpy array primitives (elementwise ops, matmul, bincount) and no blocking,
fusion or reordering of its own:

  locate            Section 3.4 (the level-l cell that contains x)
  octa_encode       Section 3.3, Eq. 4 (projection) and Eq. 5 (fold)
  octa_decode       inverse of Eq. 4/5 (used only by the pins)
  corner_base_f32   canonical binary32 form of Eq. 4/5 + texel lookup,
                    which fixes the integer texel coordinates
  wrap              octahedral edge wrap of the texel grid (Section 3.3: the
                    map is continuous across the unfolded edges)
  encode_features   Eq. 10 in the single-cell, bilinear form + Eq. 11
  encode_features_full  Eq. 10 as printed (eight cells, renormalised
                    trilinear weights) with Eq. 6 (barycentric on vertex maps)
  encode_features_shifted  the same with Eq. 7-9's disparity-shifted
                    direction per cell (reflect_f32, shifted_direction_f32)
  hash_encode, disparity  the predictor g_psi of Eq. 7 (Section 3.5): a
                    multiresolution hash encoding of x (Mueller et al. 2022)
                    and a bias-free ReLU MLP on [encoding, omega_r], exp out
  shifted_features_d_gradient, disparity_backward  training g_psi: the
                    features' derivative with respect to d and g_psi's
                    gradients
  disparity_gradient  dL/dd of a query through the shifted lookup (Eq. 7-9)
  shifted_train_gradients  a whole training step's gradients in the shifted
                    form with the predicted disparity (Eq. 7-9, 14; Section
                    3.3: d learnt only through the radiance objective)
  mlp_forward       Eq. 13 (decoder; ReLU hidden layers, exp output)
  residual_loss     Eq. 14 with the Monte-Carlo target of Eq. 3 (M = 1)
  residual_loss_multi  Eq. 14 with Eq. 3's M-sample target
  trace_rays_f32    Eq. 2's first intersection x'(omega_i) with the synthetic
                    scene (planes, spheres, the box's inner walls), every
                    decision in binary32 in a fixed operation order
  quarter_schedule  Section 4: halve the LHS count and double M after each
                    quarter of the schedule
  query_backward    derivative of Eq. 13, then of Eq. 10/11 w.r.t. the table
  adam_update       Kingma & Ba (2015), with bias correction
  LossScaler        dynamic loss scaling, Micikevicius et al. (2018)
  build_tree        seeded octree (SplitMix64, Steele et al. 2014)

Readings where the paper is silent (sign(0) = +1, the wrap rule, eps = 1e-2,
no decoder biases, Adam hyper-parameters, the tree generator) are listed in
the design notes.  Every function here is pinned by a CPU test against a
closed form, a brute-force search, an invariant or finite differences.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1


# ---------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014), written from its published definition.
# ---------------------------------------------------------------------------

def splitmix64_next(state):
    """Advance the state by the golden gamma and return (state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def splitmix64_unit(z):
    """Top 53 bits of an output as a double in [0, 1)."""
    return (z >> 11) * (2.0 ** -53)


# ---------------------------------------------------------------------------
# Octree (Section 3.4: a multi-level sparse octree; every non-empty cell of
# every level stores an octahedral map).
# ---------------------------------------------------------------------------

@dataclass
class Tree:
    first_child: np.ndarray       # [num_nodes] int64, -1 = leaf
    node_coord: np.ndarray        # [num_nodes][3] int64, integer cell coords at its level
    node_level: np.ndarray        # [num_nodes] int64
    level_node_start: np.ndarray  # [K+1]
    level_texel_base: np.ndarray  # [K+1]
    map_offset: np.ndarray        # [num_nodes] int64, texel index of texel (0,0)
    R: list                       # map side per level

    @property
    def num_levels(self):
        return len(self.R)

    @property
    def num_nodes(self):
        return len(self.first_child)

    @property
    def num_texels(self):
        return int(self.level_texel_base[-1])


def _finish_tree(first_child, coords, levels, R):
    K = len(R)
    first_child = np.asarray(first_child, dtype=np.int64)
    coords = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
    levels = np.asarray(levels, dtype=np.int64)
    n = len(levels)
    start = np.empty(K + 1, dtype=np.int64)
    for l in range(K + 1):
        # first node whose level is >= l (levels are non-decreasing in BFS order)
        start[l] = int(np.searchsorted(levels, l, side="left"))
    start[K] = n
    base = np.zeros(K + 1, dtype=np.int64)
    for l in range(K):
        base[l + 1] = base[l] + (start[l + 1] - start[l]) * R[l] * R[l]
    offs = np.empty(n, dtype=np.int64)
    for i in range(n):
        l = levels[i]
        offs[i] = base[l] + (i - start[l]) * R[l] * R[l]
    return Tree(first_child, coords, levels, start, base, offs, list(R))


def _bfs_tree(decide, max_depth, R):
    """Breadth-first construction; decide(node_index, depth) -> subdivide?"""
    coords = [(0, 0, 0)]
    levels = [0]
    first_child = []
    i = 0
    while i < len(coords):
        d = levels[i]
        if d < max_depth and decide(i, d):
            first_child.append(len(coords))
            cx, cy, cz = coords[i]
            for b in range(8):            # child slot b = bx | by<<1 | bz<<2
                coords.append((2 * cx + (b & 1), 2 * cy + ((b >> 1) & 1), 2 * cz + ((b >> 2) & 1)))
                levels.append(d + 1)
        else:
            first_child.append(-1)
        i += 1
    return _finish_tree(first_child, coords, levels, R)


def build_tree(seed, max_depth, p_base, R):
    """Seeded probabilistic octree: a node at depth d < max_depth draws one
    SplitMix64 uniform (in node order) and splits iff u < p_base^d, where
    p_base^d is the product of d factors p_base taken left to right from 1."""
    assert len(R) == max_depth + 1
    thr = [1.0]
    for _ in range(max_depth):
        thr.append(thr[-1] * p_base)
    st = [seed & MASK64]

    def decide(i, d):
        st[0], z = splitmix64_next(st[0])
        return splitmix64_unit(z) < thr[d]

    return _bfs_tree(decide, max_depth, R)


def tree_from_flags(flags, max_depth, R):
    """Hand-written tree: flags[k] decides the k-th node (in node order) whose
    depth is below max_depth; missing flags mean 'leaf'."""
    k = [0]

    def decide(i, d):
        j = k[0]
        k[0] += 1
        return j < len(flags) and bool(flags[j])

    return _bfs_tree(decide, max_depth, R)


def table_entries(node_counts, sides):
    """Storage accounting: sum over levels of nodes x (map side)^2."""
    return int(sum(int(n) * int(s) * int(s) for n, s in zip(node_counts, sides)))


# ---------------------------------------------------------------------------
# Point location (Section 3.4; single containing cell per level)
# ---------------------------------------------------------------------------

def cell_coords(x, l):
    """Integer coordinates of the level-l cell containing x (clamped to [0,1];
    cells are half-open and x = 1 falls in the last cell)."""
    x64 = np.clip(np.asarray(x, dtype=np.float64), 0.0, 1.0)
    n = 1 << l
    return np.minimum(np.floor(x64 * n), n - 1).astype(np.int64)


def locate(tree, x):
    """Node index per level [N][K] by descent from the root; -1 below a leaf."""
    N = len(x)
    K = tree.num_levels
    out = np.full((N, K), -1, dtype=np.int64)
    node = np.zeros(N, dtype=np.int64)
    out[:, 0] = 0
    c_prev = cell_coords(x, 0)
    for l in range(1, K):
        c = cell_coords(x, l)
        b = c - 2 * c_prev
        slot = b[:, 0] | (b[:, 1] << 1) | (b[:, 2] << 2)
        alive = node >= 0
        fc = np.where(alive, tree.first_child[np.maximum(node, 0)], -1)
        node = np.where(fc >= 0, fc + slot, -1)
        out[:, l] = node
        c_prev = c
    return out


def locate_bruteforce(tree, x):
    """Scan every node of level l for the one whose cell holds x."""
    N = len(x)
    K = tree.num_levels
    out = np.full((N, K), -1, dtype=np.int64)
    for l in range(K):
        c = cell_coords(x, l)
        lo, hi = tree.level_node_start[l], tree.level_node_start[l + 1]
        for n in range(lo, hi):
            hit = np.all(c == tree.node_coord[n], axis=1)
            out[hit, l] = n
    return out


# ---------------------------------------------------------------------------
# Octahedral map (Section 3.3, Eq. 4 and Eq. 5)
# ---------------------------------------------------------------------------

def _sgn(a):
    """sign with sign(0) = +1 (the paper leaves sign(0) open)."""
    return np.where(a >= 0, 1.0, -1.0)


def octa_encode(omega):
    """Eq. 4 then Eq. 5: omega [N][3] -> u [N][2] in [-1,1]^2 (FP64)."""
    w = np.asarray(omega, dtype=np.float64)
    s = np.abs(w[:, 0]) + np.abs(w[:, 1]) + np.abs(w[:, 2])
    ux = w[:, 0] / s
    uy = w[:, 1] / s
    lower = w[:, 2] < 0
    fx = (1.0 - np.abs(uy)) * _sgn(ux)
    fy = (1.0 - np.abs(ux)) * _sgn(uy)
    return np.stack([np.where(lower, fx, ux), np.where(lower, fy, uy)], axis=1)


def octa_uv(omega):
    """Eq. 4/5 remapped to [0,1]^2."""
    return (octa_encode(omega) + 1.0) * 0.5


def octa_decode(u):
    """Inverse of Eq. 4/5 on [-1,1]^2 -> unit direction."""
    u = np.asarray(u, dtype=np.float64)
    ux, uy = u[:, 0], u[:, 1]
    z = 1.0 - np.abs(ux) - np.abs(uy)
    lower = z < 0
    fx = (1.0 - np.abs(uy)) * _sgn(ux)
    fy = (1.0 - np.abs(ux)) * _sgn(uy)
    vx = np.where(lower, fx, ux)
    vy = np.where(lower, fy, uy)
    v = np.stack([vx, vy, z], axis=1)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def corner_base_f32(omega32, R):
    """Integer texel corner (i0, j0) from the canonical binary32 sequence.

    Eq. 4/5 evaluated in IEEE binary32, round-to-nearest-even, one rounding
    per operation (numpy float32 ufuncs, no fused multiply-add):
      s = (|wx| + |wy|) + |wz|;  u = (wx / s, wy / s);  fold if wz < 0;
      uv = u * 0.5 + 0.5;  p = uv * R - 0.5;  (i0, j0) = floor(p).
    Texel (i, j) is centred at ((i + 1/2)/R, (j + 1/2)/R); i runs along u_x.
    """
    f = np.float32
    w = np.asarray(omega32, dtype=np.float32)
    ax, ay, az = np.abs(w[:, 0]), np.abs(w[:, 1]), np.abs(w[:, 2])
    s = (ax + ay) + az
    ux = w[:, 0] / s
    uy = w[:, 1] / s
    one = f(1.0)
    sx = np.where(ux >= 0, one, -one).astype(np.float32)
    sy = np.where(uy >= 0, one, -one).astype(np.float32)
    fx = (one - np.abs(uy)) * sx
    fy = (one - np.abs(ux)) * sy
    lower = w[:, 2] < 0
    ux = np.where(lower, fx, ux).astype(np.float32)
    uy = np.where(lower, fy, uy).astype(np.float32)
    px = (ux * f(0.5) + f(0.5)) * f(R) - f(0.5)
    py = (uy * f(0.5) + f(0.5)) * f(R) - f(0.5)
    assert px.dtype == np.float32 and py.dtype == np.float32
    return np.floor(px).astype(np.int64), np.floor(py).astype(np.int64)


def wrap(i, j, R):
    """Octahedral wrap of a corner in [-1, R]^2 onto the R x R grid.

    Across the edge u_x = +-1 the map continues mirrored in u_y, across
    u_y = +-1 mirrored in u_x (the lower-hemisphere fold of Eq. 5 glues the
    square's edges this way); applied to i first, then to j.
    """
    i = np.asarray(i, dtype=np.int64).copy()
    j = np.asarray(j, dtype=np.int64).copy()
    lo = i == -1
    hi = i == R
    j = np.where(lo | hi, R - 1 - j, j)
    i = np.where(lo, 0, np.where(hi, R - 1, i))
    lo = j == -1
    hi = j == R
    i = np.where(lo | hi, R - 1 - i, i)
    j = np.where(lo, 0, np.where(hi, R - 1, j))
    return i, j


@dataclass
class Encoding:
    h: np.ndarray           # [N][K*F] FP64 concatenated features (Eq. 11)
    node: np.ndarray        # [N][K] node index per level (-1 absent)
    addr: np.ndarray        # [N][K][4] texel index per corner (-1 absent)
    weight: np.ndarray      # [N][K][4] FP64 bilinear weights (0 where absent)


def encode_features(tree, tables, x, omega):
    """Per level: containing node, octahedral texel lookup, bilinear blend of
    the 4 surrounding texels; levels concatenated (Eq. 10 single-cell form,
    Eq. 11).  An absent cell contributes zero features (the indicator of
    Eq. 10).  Corner order k = a + 2b for corner (i0 + a, j0 + b)."""
    T = np.asarray(tables, dtype=np.float64)
    F = T.shape[1]
    N = len(x)
    K = tree.num_levels
    node = locate(tree, x)
    uv = octa_uv(np.asarray(omega, dtype=np.float32).astype(np.float64))
    h = np.zeros((N, K * F))
    addr = np.full((N, K, 4), -1, dtype=np.int64)
    wgt = np.zeros((N, K, 4))
    for l in range(K):
        R = tree.R[l]
        i0, j0 = corner_base_f32(omega, R)
        fx = uv[:, 0] * R - 0.5 - i0
        fy = uv[:, 1] * R - 0.5 - j0
        w4 = [(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy]
        present = node[:, l] >= 0
        base = np.where(present, tree.map_offset[np.maximum(node[:, l], 0)], 0)
        for k in range(4):
            ci, cj = wrap(i0 + (k & 1), j0 + (k >> 1), R)
            a = base + cj * R + ci
            addr[:, l, k] = np.where(present, a, -1)
            wgt[:, l, k] = np.where(present, w4[k], 0.0)
            h[:, l * F:(l + 1) * F] += wgt[:, l, k][:, None] * T[np.where(present, a, 0)] \
                * present[:, None]
    return Encoding(h, node, addr, wgt)


# ---------------------------------------------------------------------------
# The full query (Section 3.3 Eq. 6, Section 3.4 Eq. 10): directional
# features stored at map vertices and interpolated barycentrically over the
# triangle holding the direction, spatial features blended over the eight
# cells around x with trilinear weights renormalised over non-empty cells
# ---------------------------------------------------------------------------

def node_of_cell(tree, l, c):
    """Node of the level-l cell c [N][3] (descent from the root along the
    cell's ancestors), -1 where the cell is not in the octree."""
    c = np.asarray(c, dtype=np.int64)
    node = np.zeros(len(c), dtype=np.int64)
    for m in range(1, l + 1):
        b = (c >> (l - m)) & 1
        slot = b[:, 0] | (b[:, 1] << 1) | (b[:, 2] << 2)
        fc = np.where(node >= 0, tree.first_child[np.maximum(node, 0)], -1)
        node = np.where(fc >= 0, fc + slot, -1)
    return node


def node_of_cell_bruteforce(tree, l, c):
    """Scan every node of level l for cell c."""
    c = np.asarray(c, dtype=np.int64)
    out = np.full(len(c), -1, dtype=np.int64)
    for n in range(tree.level_node_start[l], tree.level_node_start[l + 1]):
        out[np.all(c == tree.node_coord[n], axis=1)] = n
    return out


def neighbour_cells(x, l):
    """The eight level-l cells whose centres surround x, with standard
    trilinear weights.  Cell k has centre (k + 1/2) / 2^l; the lower corner
    cell is c0 = floor(p) with p = x 2^l - 1/2 evaluated in binary32 (the
    integer decision is taken in the kernel's precision; x 2^l is exact and
    the subtraction rounds at most once), the weights in FP64.  Neighbour j
    is c0 + (j & 1, (j >> 1) & 1, j >> 2).  Returns cells [N][8][3], weights
    [N][8] and whether each cell lies inside the cube [N][8]."""
    f = np.float32
    n = 1 << l
    x32 = np.clip(np.asarray(x, dtype=np.float32), f(0.0), f(1.0))
    p32 = x32 * f(n) - f(0.5)
    c0 = np.floor(p32).astype(np.int64)
    t = x32.astype(np.float64) * n - 0.5 - c0
    cells = np.zeros((len(x32), 8, 3), dtype=np.int64)
    wts = np.ones((len(x32), 8))
    for j in range(8):
        d = np.array([j & 1, (j >> 1) & 1, j >> 2])
        cells[:, j, :] = c0 + d
        for a in range(3):
            wts[:, j] *= t[:, a] if d[a] else 1.0 - t[:, a]
    inside = np.all((cells >= 0) & (cells < n), axis=2)
    return cells, wts, inside


def vertex_cell_f32(omega32, V):
    """Grid cell (i0, j0) of a V x V vertex map (N = V - 1 cells a side;
    vertex (i, j) sits at uv = (i, j) / N) and the fractions (fx, fy) inside
    it, from the canonical binary32 sequence of corner_base_f32 with
    p = uv * N (no half-texel shift): (i0, j0) = min(floor(p), N - 1),
    f = p - (i0, j0) (exact in binary32).  Returns float32 fractions."""
    f = np.float32
    w = np.asarray(omega32, dtype=np.float32)
    ax, ay, az = np.abs(w[:, 0]), np.abs(w[:, 1]), np.abs(w[:, 2])
    s = (ax + ay) + az
    ux = w[:, 0] / s
    uy = w[:, 1] / s
    one = f(1.0)
    sx = np.where(ux >= 0, one, -one).astype(np.float32)
    sy = np.where(uy >= 0, one, -one).astype(np.float32)
    fx = (one - np.abs(uy)) * sx
    fy = (one - np.abs(ux)) * sy
    lower = w[:, 2] < 0
    ux = np.where(lower, fx, ux).astype(np.float32)
    uy = np.where(lower, fy, uy).astype(np.float32)
    N = V - 1
    px = (ux * f(0.5) + f(0.5)) * f(N)
    py = (uy * f(0.5) + f(0.5)) * f(N)
    i0 = np.minimum(np.floor(px), f(N - 1)).astype(np.int64)
    j0 = np.minimum(np.floor(py), f(N - 1)).astype(np.int64)
    return i0, j0, (px - i0.astype(np.float32)).astype(np.float32), \
        (py - j0.astype(np.float32)).astype(np.float32)


def vertex_triangle(i0, j0, fx32, fy32, N):
    """The right isosceles triangle of cell (i0, j0) that holds the point,
    as three vertex offsets (da, db) and the barycentric weights (Eq. 6).

    Each octahedron face is tiled by the unfolded triangles, so a cell is
    split along the diagonal parallel to its quadrant's face boundary
    (|u_x| + |u_y| = 1): the anti-diagonal in the quadrants u_x, u_y of equal
    sign, the main diagonal otherwise (N is even, so no cell straddles a
    quadrant edge).  The side of the diagonal is decided in binary32
    (fx + fy <= 1, or fy <= fx); the weights are those of the FP64
    fractions.  Returns offsets [N][3][2] and weights [N][3]."""
    f = np.float32
    fx = fx32.astype(np.float64)
    fy = fy32.astype(np.float64)
    anti = (i0 >= N // 2) == (j0 >= N // 2)
    a_lower = (fx32 + fy32) <= f(1.0)
    m_lower = fy32 <= fx32
    n = len(i0)
    off = np.zeros((n, 3, 2), dtype=np.int64)
    b = np.zeros((n, 3))
    # anti-diagonal, lower-left triangle (0,0) (1,0) (0,1)
    m = anti & a_lower
    off[m] = [[0, 0], [1, 0], [0, 1]]
    b[m] = np.stack([1 - fx - fy, fx, fy], 1)[m]
    # anti-diagonal, upper-right triangle (1,1) (1,0) (0,1)
    m = anti & ~a_lower
    off[m] = [[1, 1], [1, 0], [0, 1]]
    b[m] = np.stack([fx + fy - 1, 1 - fy, 1 - fx], 1)[m]
    # main diagonal, lower-right triangle (0,0) (1,0) (1,1)
    m = ~anti & m_lower
    off[m] = [[0, 0], [1, 0], [1, 1]]
    b[m] = np.stack([1 - fx, fx - fy, fy], 1)[m]
    # main diagonal, upper-left triangle (0,0) (0,1) (1,1)
    m = ~anti & ~m_lower
    off[m] = [[0, 0], [0, 1], [1, 1]]
    b[m] = np.stack([1 - fy, fy - fx, fx], 1)[m]
    return off, b


def canonical_vertex(i, j, N):
    """One representative of each vertex of the unfolded map.  The fold of
    Eq. 5 glues each edge of the square to itself mirrored: (N, j) and
    (0, j) are the directions of (N, N - j) and (0, N - j), (i, N) and (i, 0)
    those of (N - i, N) and (N - i, 0); the four corners are one direction.
    Vertical edges first (j -> min(j, N - j)), then horizontal edges
    (i -> min(i, N - i))."""
    i = np.asarray(i, dtype=np.int64).copy()
    j = np.asarray(j, dtype=np.int64).copy()
    v = (i == 0) | (i == N)
    j = np.where(v, np.minimum(j, N - j), j)
    hz = (j == 0) | (j == N)
    i = np.where(hz, np.minimum(i, N - i), i)
    return i, j


@dataclass
class FullEncoding:
    h: np.ndarray           # [N][K*F] FP64 features (Eq. 10 with Eq. 6, Eq. 11)
    addr: np.ndarray        # [N][K][8][3] vertex entry per neighbour and vertex (-1 absent)
    weight: np.ndarray      # [N][K][8][3] FP64 weight (renormalised trilinear x barycentric)


def encode_features_full(tree, tables, x, omega):
    """Eq. 10 as printed, with the directional lookup of Eq. 6 and without
    the disparity shift (the same direction omega in all eight cells): per
    level, the eight cells around x with trilinear weights renormalised over
    the cells present in the octree (a level with none gives zero features),
    in each the barycentric blend of the three vertex features of the
    triangle holding omega on that node's V x V vertex map (V = R[l]);
    levels concatenated (Eq. 11).  Vertex (i, j) of a node's map is entry
    map_offset + j V + i of the canonical representative (i, j)."""
    T = np.asarray(tables, dtype=np.float64)
    F = T.shape[1]
    n = len(x)
    K = tree.num_levels
    om32 = np.asarray(omega, dtype=np.float32)
    h = np.zeros((n, K * F))
    addr = np.full((n, K, 8, 3), -1, dtype=np.int64)
    wgt = np.zeros((n, K, 8, 3))
    for l in range(K):
        V = int(tree.R[l])
        N = V - 1
        cells, wsp, inside = neighbour_cells(x, l)
        nodes = np.full((n, 8), -1, dtype=np.int64)
        for j in range(8):
            nodes[:, j] = np.where(inside[:, j], node_of_cell(tree, l, np.clip(cells[:, j], 0, None)), -1)
        present = nodes >= 0
        wp = np.where(present, wsp, 0.0)
        den = wp.sum(axis=1)
        wn = np.where(den[:, None] > 0, wp / np.where(den > 0, den, 1.0)[:, None], 0.0)
        i0, j0, fx32, fy32 = vertex_cell_f32(om32, V)
        off, b = vertex_triangle(i0, j0, fx32, fy32, N)
        for k in range(3):
            vi, vj = canonical_vertex(i0 + off[:, k, 0], j0 + off[:, k, 1], N)
            vidx = vj * V + vi
            for j in range(8):
                base = tree.map_offset[np.maximum(nodes[:, j], 0)]
                a = np.where(present[:, j], base + vidx, -1)
                w = wn[:, j] * b[:, k]
                addr[:, l, j, k] = a
                wgt[:, l, j, k] = np.where(present[:, j], w, 0.0)
                h[:, l * F:(l + 1) * F] += (wgt[:, l, j, k][:, None] * T[np.maximum(a, 0)]
                                            * present[:, j][:, None])
    return FullEncoding(h, addr, wgt)


def reflect_f32(omega, normal):
    """The mirror reflection direction omega_r of Eq. 7 in binary32, one
    rounding per operation: omega and n normalised (v / sqrt(v.v)), then
    omega_r = (2 (n.omega)) n - omega per component; dot products
    ((a0 b0 + a1 b1) + a2 b2)."""
    f = np.float32

    def dot(a, b):
        return ((a[:, 0] * b[:, 0]).astype(f) + (a[:, 1] * b[:, 1]).astype(f)).astype(f) + \
            (a[:, 2] * b[:, 2]).astype(f)

    def unit(v):
        v = np.asarray(v, dtype=f)
        return (v / np.sqrt(dot(v, v)).astype(f)[:, None]).astype(f)
    w = unit(omega)
    n = unit(normal)
    d2 = (f(2) * dot(n, w)).astype(f)
    return ((d2[:, None] * n).astype(f) - w).astype(f)


def shifted_direction_f32(x, omega_r, disparity, cells, l):
    """Eq. 9's direction in the cell with integer coordinates `cells` [N][3]
    at level l, in binary32 with one rounding per operation:
    v = (x - c) d + omega_r per component, c = (cell + 1/2) 2^-l (exact).
    The normalisation of Eq. 9 is left out: the octahedral map of Eq. 4
    divides by the L1 norm, so v and v / |v| fold to the same point."""
    f = np.float32
    x32 = np.clip(np.asarray(x, dtype=f), f(0), f(1))
    c = ((cells.astype(f) + f(0.5)) * f(2.0 ** -l)).astype(f)
    d = np.asarray(disparity, dtype=f)[:, None]
    return (((x32 - c).astype(f) * d).astype(f) + np.asarray(omega_r, dtype=f)).astype(f)


def encode_features_shifted(tree, tables, x, omega, normal, disparity):
    """Eq. 10 with the disparity-shifted lookup of Eq. 7-9 and Eq. 6: as
    encode_features_full, but cell j of level l looks its vertex map up in
    the direction of y - c_j, y = x + omega_r / d (Eq. 8), i.e. of
    (x - c_j) d + omega_r (Eq. 9), with omega_r the reflection of omega
    about the normal (Eq. 7) and d the given disparity per query.  d = 0
    looks every cell up at omega_r."""
    T = np.asarray(tables, dtype=np.float64)
    F = T.shape[1]
    n = len(x)
    K = tree.num_levels
    om_r = reflect_f32(omega, normal)
    h = np.zeros((n, K * F))
    addr = np.full((n, K, 8, 3), -1, dtype=np.int64)
    wgt = np.zeros((n, K, 8, 3))
    for l in range(K):
        V = int(tree.R[l])
        N = V - 1
        cells, wsp, inside = neighbour_cells(x, l)
        nodes = np.full((n, 8), -1, dtype=np.int64)
        for j in range(8):
            nodes[:, j] = np.where(inside[:, j], node_of_cell(tree, l, np.clip(cells[:, j], 0, None)), -1)
        present = nodes >= 0
        wp = np.where(present, wsp, 0.0)
        den = wp.sum(axis=1)
        wn = np.where(den[:, None] > 0, wp / np.where(den > 0, den, 1.0)[:, None], 0.0)
        for j in range(8):
            v = shifted_direction_f32(x, om_r, disparity, cells[:, j], l)
            i0, j0, fx32, fy32 = vertex_cell_f32(v, V)
            off, b = vertex_triangle(i0, j0, fx32, fy32, N)
            base = tree.map_offset[np.maximum(nodes[:, j], 0)]
            for k in range(3):
                vi, vj = canonical_vertex(i0 + off[:, k, 0], j0 + off[:, k, 1], N)
                a = np.where(present[:, j], base + vj * V + vi, -1)
                w = np.where(present[:, j], wn[:, j] * b[:, k], 0.0)
                addr[:, l, j, k] = a
                wgt[:, l, j, k] = w
                h[:, l * F:(l + 1) * F] += w[:, None] * T[np.maximum(a, 0)] * present[:, j][:, None]
    return FullEncoding(h, addr, wgt)


# ---------------------------------------------------------------------------
# Decoder (Section 3.5, Eq. 13): bias-free MLP, ReLU hidden, exp output
# ---------------------------------------------------------------------------

def mlp_forward(weights, h):
    """Returns (rgb, pre-activations z_i, layer inputs a_{i-1})."""
    Ws = [np.asarray(W, dtype=np.float64) for W in weights]
    a = np.asarray(h, dtype=np.float64)
    inputs, zs = [], []
    for i, W in enumerate(Ws):
        inputs.append(a)
        z = a @ W.T
        zs.append(z)
        if i < len(Ws) - 1:
            a = np.maximum(z, 0.0)
    return np.exp(zs[-1]), zs, inputs


FORMS = ("cell", "full")


def _encode(tree, tables, x, omega, form, normal=None, disparity=None):
    """Encoding in the query form: "cell" (encode_features), "full"
    (encode_features_full) or "shifted" (encode_features_shifted, with the
    normal and disparity); returns (h, addr [N][K][n_entries],
    weight [N][K][n_entries])."""
    if form == "cell":
        e = encode_features(tree, tables, x, omega)
        return e, e.h, e.addr, e.weight
    if form in ("full", "shifted"):
        if form == "full":
            e = encode_features_full(tree, tables, x, omega)
        else:
            e = encode_features_shifted(tree, tables, x, omega, normal, disparity)
        n, K = e.h.shape[0], tree.num_levels
        return e, e.h, e.addr.reshape(n, K, 24), e.weight.reshape(n, K, 24)
    raise ValueError(form)


def decoder_input(h, attrs):
    """Eq. 12: the decoder sees [h, g], the per-query surface attributes g
    (position, reflection direction, normal, albedo, roughness in the paper)
    appended after the K F features; attrs None: h alone."""
    if attrs is None:
        return h
    return np.concatenate([h, np.asarray(attrs, dtype=np.float64)], axis=1)


def query_forward(tree, tables, weights, x, omega, form="cell", normal=None, disparity=None,
                  attrs=None):
    """L_hat(x, omega) = f_phi(h, g) (Eq. 13): encoding, the attributes of
    Eq. 12 when given, then decoder.  Returns (rgb, encoding)."""
    enc, h, _, _ = _encode(tree, tables, x, omega, form, normal, disparity)
    rgb, _, _ = mlp_forward(weights, decoder_input(h, attrs))
    return rgb, enc


# ---------------------------------------------------------------------------
# Training objective (Section 3.2 Eq. 3, Section 3.6 Eq. 14)
# ---------------------------------------------------------------------------

def residual_loss(Lp, Ls, E, w, eps=1e-2, rhs_grad=True, scale=1.0):
    """Relative L2 between L_hat(x, omega) and the one-sample RHS
    T = E + w * L_hat(x', -omega') (Eq. 3 with M = 1, w = f_r |n.omega'| / p).
    The normaliser sg[L_hat + T + eps] is detached (Eq. 14).  With rhs_grad
    the gradient also flows into L_hat(x', -omega') through T in the
    numerator; without it T is detached as in Eq. 14.  The loss averages the
    per-channel squares over pairs and channels.  Gradients are for
    scale * loss."""
    Lp = np.asarray(Lp, dtype=np.float64)
    Ls = np.asarray(Ls, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    T = E + w * Ls
    den = Lp + T + eps
    r = (Lp - T) / den
    n = Lp.size
    loss = float(np.sum(r * r) / n)
    dLp = scale * 2.0 * r / (n * den)
    dLs = -scale * 2.0 * r * w / (n * den) if rhs_grad else np.zeros_like(Ls)
    return loss, dLp, dLs


def query_backward(tree, tables, weights, x, omega, d_rgb, form="cell", attrs=None, normal=None,
                   disparity=None, return_dh=False):
    """Gradients of sum(d_rgb * L_hat) w.r.t. the table and the weights.

    Decoder: delta_L = d_rgb * exp(z_L); dW_i = delta_i^T a_{i-1};
    delta_{i-1} = (delta_i W_i) * 1[z_{i-1} > 0]; dh = delta_1 W_1.
    Encoding: each present entry k of level l (4 corners in the cell form,
    8 cells x 3 vertices in the full form) receives weight_k * dh_l.
    Returns (dT, dWs, rgb), and the decoder-input gradient dh [N][width]
    as a fourth value when return_dh.
    """
    T = np.asarray(tables, dtype=np.float64)
    F = T.shape[1]
    K = tree.num_levels
    _, h, addr, weight = _encode(tree, T, x, omega, form, normal, disparity)
    rgb, zs, inputs = mlp_forward(weights, decoder_input(h, attrs))
    Ws = [np.asarray(W, dtype=np.float64) for W in weights]
    delta = np.asarray(d_rgb, dtype=np.float64) * rgb
    dWs = [None] * len(Ws)
    for i in range(len(Ws) - 1, -1, -1):
        dWs[i] = delta.T @ inputs[i]
        g = delta @ Ws[i]
        if i > 0:
            delta = g * (zs[i - 1] > 0)
        else:
            dh = g
    dT = np.zeros_like(T)
    for l in range(K):
        for k in range(addr.shape[2]):
            a = addr[:, l, k]
            ok = a >= 0
            for f in range(F):
                dT[:, f] += np.bincount(a[ok], weights=weight[ok, l, k] * dh[ok, l * F + f],
                                        minlength=len(T))
    if return_dh:
        return dT, dWs, rgb, dh
    return dT, dWs, rgb


def surrogate_loss(tree, tables, weights, pairs_x, pairs_w, x2, w2neg, E, w, D0, T0, eps, rhs_grad):
    """Eq. 14 with its stop-gradients made explicit: the normaliser (and the
    target when rhs_grad is off) frozen at their values D0, T0.  Central
    finite differences of this function equal the analytic gradient."""
    Lp, _ = query_forward(tree, tables, weights, pairs_x, pairs_w)
    if rhs_grad:
        Ls, _ = query_forward(tree, tables, weights, x2, w2neg)
        T = np.asarray(E, np.float64) + np.asarray(w, np.float64) * Ls
    else:
        T = T0
    r = (Lp - T) / (D0 + eps)
    return float(np.sum(r * r) / Lp.size)


# ---------------------------------------------------------------------------
# Optimiser (paper silent; Adam, Kingma & Ba 2015) and loss scaling
# (Micikevicius et al. 2018)
# ---------------------------------------------------------------------------

def adam_update(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step at step number t >= 1 with bias correction."""
    p = np.asarray(p, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


class LossScaler:
    """Dynamic loss scale: gradients are computed for S * loss and divided by
    S; a non-finite gradient skips the step and halves S; after
    growth_interval consecutive finite steps S doubles."""

    def __init__(self, scale=2.0 ** 15, growth_interval=2000):
        self.scale = float(scale)
        self.growth_interval = growth_interval
        self.good = 0

    def update(self, finite):
        """Returns True when the optimiser step must be skipped."""
        if not finite:
            self.scale *= 0.5
            self.good = 0
            return True
        self.good += 1
        if self.good == self.growth_interval:
            self.scale *= 2.0
            self.good = 0
        return False


@dataclass
class TrainState:
    tables: np.ndarray
    weights: list
    m_t: np.ndarray
    v_t: np.ndarray
    m_w: list
    v_w: list
    step: int = 0


def train_step(tree, state, pairs, scaler=None, eps=1e-2, rhs_grad=True,
               lr_tables=1e-2, lr_mlp=1e-3):
    """One step: queries at (x, omega) and (x', -omega') (Eq. 2 gives the
    sign), Eq. 14 loss, backward, unscale, non-finite check, Adam.
    Returns (loss, grad_norm, skipped)."""
    N = len(pairs.x)
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    rgb, _ = query_forward(tree, state.tables, state.weights, X, Om)
    S = scaler.scale if scaler is not None else 1.0
    loss, dLp, dLs = residual_loss(rgb[:N], rgb[N:], pairs.E, pairs.w, eps, rhs_grad, S)
    dT, dWs, _ = query_backward(tree, state.tables, state.weights, X, Om,
                                np.concatenate([dLp, dLs]))
    dT = dT / S
    dWs = [d / S for d in dWs]
    sq = float(np.sum(dT * dT)) + sum(float(np.sum(d * d)) for d in dWs)
    finite = bool(np.isfinite(sq))
    skipped = scaler.update(finite) if scaler is not None else not finite
    if not skipped:
        state.step += 1
        t = state.step
        state.tables, state.m_t, state.v_t = adam_update(state.tables, dT, state.m_t, state.v_t,
                                                         t, lr_tables)
        for i in range(len(state.weights)):
            state.weights[i], state.m_w[i], state.v_w[i] = adam_update(
                state.weights[i], dWs[i], state.m_w[i], state.v_w[i], t, lr_mlp)
    return loss, float(np.sqrt(sq)), skipped


# ---------------------------------------------------------------------------
# The paper's training regime: M RHS samples per LHS sample (Eq. 3), the
# quarter schedule (Section 4) and the secondary hits x'(omega_i) (Eq. 2)
# ---------------------------------------------------------------------------

def rhs_target(E, w, Ls):
    """Eq. 3: T = E + (1/M) sum_m w_m * L_hat(x'^m, -omega_i^m), with
    w_m = f_r |n . omega_i^m| / p(omega_i^m).  E [N][3]; w, Ls [N][M][3]."""
    E = np.asarray(E, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    Ls = np.asarray(Ls, dtype=np.float64)
    M = w.shape[1]
    return E + np.sum(w * Ls, axis=1) / M


def residual_loss_multi(Lp, Ls, E, w, eps=1e-2, rhs_grad=True, scale=1.0):
    """Eq. 14 against the M-sample target of Eq. 3.  Lp, E [N][3]; Ls, w
    [N][M][3].  The normaliser is detached; with rhs_grad the gradient flows
    into every secondary radiance through T (dT/dLs_m = w_m / M), without it
    the target is detached as Eq. 14 prints.  Returns (loss, dLp [N][3],
    dLs [N][M][3]), gradients of scale * loss; loss = mean over 3N."""
    Lp = np.asarray(Lp, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    M = w.shape[1]
    T = rhs_target(E, w, Ls)
    den = Lp + T + eps
    r = (Lp - T) / den
    n = Lp.size
    loss = float(np.sum(r * r) / n)
    dLp = scale * 2.0 * r / (n * den)
    if rhs_grad:
        dLs = -(dLp[:, None, :] * w) / M
    else:
        dLs = np.zeros(w.shape)
    return loss, dLp, dLs


def quarter_schedule(step, total_steps, n0, m0, quarters=4):
    """(LHS samples, M) of a 0-based step: after every quarter of the
    schedule the LHS count halves and M doubles (Section 4)."""
    q = min(quarters - 1, (quarters * step) // total_steps)
    return n0 >> q, m0 << q


def _dot3_f32(a, b):
    """((a0 b0 + a1 b1) + a2 b2) in binary32, one rounding per operation."""
    f = np.float32
    return ((a[..., 0] * b[..., 0]).astype(f) + (a[..., 1] * b[..., 1]).astype(f)).astype(f) + \
        (a[..., 2] * b[..., 2]).astype(f)


def trace_rays_f32(planes, spheres, o, d, t_min):
    """First intersection of each ray o + t d (t > t_min) with the scene, in
    binary32 with one rounding per operation in the order written here, so
    the hit primitive, t and the point are fixed bit for bit.

    planes [P][13]: point p, unit normal n, tangents t1, t2, half-size h
    (the square patch |(x - p).t1| <= h, |(x - p).t2| <= h; inf: unbounded);
    spheres [S][4]: centre c, radius r; then the box's six inner walls
    (x_a = 0, x_a = 1 for a = 0, 1, 2).  Primitive ids: planes 0..P-1,
    spheres P..P+S-1, walls P+S + 2a + (wall == 1).  Tests run planes,
    spheres, walls in index order and replace the best hit only on a strictly
    smaller t.  Plane: t = ((p - o).n) / (d.n).  Sphere (|d| = 1 assumed):
    b = (o - c).d, disc = b^2 - ((o - c).(o - c) - r^2), t = -b - sqrt(disc)
    if that exceeds t_min, else -b + sqrt(disc).  Wall: t = (w - o_a) / d_a.
    The hit point is o + t d per component.  Returns (t [n], prim [n] int32,
    -1 and t = inf for a miss; hit [n][3]).
    """
    f = np.float32
    o = np.asarray(o, dtype=f)
    d = np.asarray(d, dtype=f)
    planes = np.asarray(planes, dtype=f).reshape(-1, 13)
    spheres = np.asarray(spheres, dtype=f).reshape(-1, 4)
    tmin = f(t_min)
    n = len(o)
    best = np.full(n, np.inf, dtype=f)
    prim = np.full(n, -1, dtype=np.int32)
    P, S = len(planes), len(spheres)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        for k in range(P):
            pk, nk, t1, t2, h = planes[k, 0:3], planes[k, 3:6], planes[k, 6:9], planes[k, 9:12], planes[k, 12]
            den = _dot3_f32(d, nk[None, :])
            num = _dot3_f32((pk[None, :] - o).astype(f), nk[None, :])
            t = (num / den).astype(f)
            hit = (o + (t[:, None] * d).astype(f)).astype(f)
            rel = (hit - pk[None, :]).astype(f)
            a = _dot3_f32(rel, t1[None, :])
            b = _dot3_f32(rel, t2[None, :])
            ok = (den != 0) & (t > tmin) & (t < best) & (np.abs(a) <= h) & (np.abs(b) <= h)
            best = np.where(ok, t, best)
            prim = np.where(ok, k, prim).astype(np.int32)
        for s_ in range(S):
            c, r = spheres[s_, 0:3], spheres[s_, 3]
            oc = (o - c[None, :]).astype(f)
            bq = _dot3_f32(oc, d)
            cq = (_dot3_f32(oc, oc) - (r * r).astype(f)).astype(f)
            disc = ((bq * bq).astype(f) - cq).astype(f)
            sq = np.sqrt(np.maximum(disc, f(0))).astype(f)
            t0 = (-bq - sq).astype(f)
            t1v = (-bq + sq).astype(f)
            t = np.where(t0 > tmin, t0, t1v).astype(f)
            ok = (disc >= 0) & (t > tmin) & (t < best)
            best = np.where(ok, t, best)
            prim = np.where(ok, P + s_, prim).astype(np.int32)
        for a in range(3):
            for wi, wall in enumerate((f(0), f(1))):
                t = ((wall - o[:, a]).astype(f) / d[:, a]).astype(f)
                ok = (t > tmin) & (t < best)
                best = np.where(ok, t, best)
                prim = np.where(ok, P + S + 2 * a + wi, prim).astype(np.int32)
        hit = (o + (best[:, None] * d).astype(f)).astype(f)
    return best, prim, hit


# ---------------------------------------------------------------------------
# The disparity predictor g_psi (Eq. 7, Section 3.5): a multiresolution hash
# encoding (Mueller, Evans, Schied & Keller 2022, written from its published
# definition) and a tiny MLP
# ---------------------------------------------------------------------------

HASH_PRIMES = (1, 2654435761, 805459861)


def hash_resolutions(levels, n_min, n_max):
    """Per-level grid resolution N_l = floor(n_min b^l), b = (n_max /
    n_min)^(1 / (levels - 1)), in FP64."""
    if levels == 1:
        return [int(n_min)]
    b = np.exp((np.log(n_max) - np.log(n_min)) / (levels - 1))
    return [int(np.floor(n_min * b ** l)) for l in range(levels)]


def hash_index(i, j, k, res, T):
    """Entry of grid vertex (i, j, k) in a level's table of T entries: the
    dense index i + j (N + 1) + k (N + 1)^2 when the (N + 1)^3 vertices fit,
    else the spatial hash (i pi_1 xor j pi_2 xor k pi_3) mod T over 32-bit
    unsigned integers."""
    side = res + 1
    i = np.asarray(i, dtype=np.uint64)
    j = np.asarray(j, dtype=np.uint64)
    k = np.asarray(k, dtype=np.uint64)
    if side ** 3 <= T:
        return (i + j * side + k * side * side).astype(np.int64)
    m = np.uint64(0xFFFFFFFF)
    h = ((i * np.uint64(HASH_PRIMES[0])) & m) ^ ((j * np.uint64(HASH_PRIMES[1])) & m) ^ \
        ((k * np.uint64(HASH_PRIMES[2])) & m)
    return (h % np.uint64(T)).astype(np.int64)


def hash_encode(table, res, x):
    """The multiresolution hash encoding of positions x [N][3] in [0, 1]:
    per level l, p = x N_l (binary32), the cell i0 = min(floor(p), N_l - 1)
    per axis, f = p - i0, and the trilinear blend (FP64 weights) of the
    features of the cell's eight vertices; levels concatenated.  table
    [L][T][F].  Returns [N][L F]."""
    tab = np.asarray(table, dtype=np.float64)
    L, T, F = tab.shape
    x32 = np.clip(np.asarray(x, dtype=np.float32), np.float32(0), np.float32(1))
    out = np.zeros((len(x32), L * F))
    for l in range(L):
        N = int(res[l])
        p = x32 * np.float32(N)
        i0 = np.minimum(np.floor(p), np.float32(N - 1)).astype(np.int64)
        f = p.astype(np.float64) - i0
        for c in range(8):
            d = np.array([c & 1, (c >> 1) & 1, c >> 2])
            idx = hash_index(i0[:, 0] + d[0], i0[:, 1] + d[1], i0[:, 2] + d[2], N, T)
            w = np.ones(len(x32))
            for a in range(3):
                w *= f[:, a] if d[a] else 1.0 - f[:, a]
            out[:, l * F:(l + 1) * F] += w[:, None] * tab[l][idx]
    return out


def disparity(table, res, weights, x, omega, normal):
    """d = g_psi(x, omega_r) (Eq. 7): the decoder-like MLP (bias-free, ReLU
    hidden, exp output, so d > 0) on [hash_encode(x), omega_r], omega_r from
    reflect_f32.  Returns d [N] (FP64)."""
    om_r = reflect_f32(omega, normal).astype(np.float64)
    inp = np.concatenate([hash_encode(table, res, x), om_r], axis=1)
    out, _, _ = mlp_forward(weights, inp)
    return out[:, 0]


# ---------------------------------------------------------------------------
# Training g_psi through the shifted lookup (Eq. 7-9): the derivative of the
# features with respect to the disparity, and g_psi's backward
# ---------------------------------------------------------------------------

def _fold_jacobian(v):
    """d(u_x, u_y)/dv of the octahedral map of Eq. 4/5 at v [N][3] (FP64,
    the branch chosen by the sign of v_z as the binary32 fold chooses it):
    upper, u = (v_x, v_y) / s with s = |v_x| + |v_y| + |v_z|, so
    du_x/dv = (e_x - u_x sgn(v)) / s; lower, u = ((1 - |b|) sgn(a),
    (1 - |a|) sgn(b)) of the upper (a, b), so du_x/dv = -sgn(a) sgn(b) db/dv
    and du_y/dv = -sgn(a) sgn(b) da/dv.  Returns [N][2][3]."""
    v = np.asarray(v, dtype=np.float64)
    s = np.abs(v).sum(axis=1)
    sg = np.where(v >= 0, 1.0, -1.0)
    a = v[:, 0] / s
    b = v[:, 1] / s
    da = (np.array([1.0, 0, 0])[None, :] - a[:, None] * sg) / s[:, None]
    db = (np.array([0, 1.0, 0])[None, :] - b[:, None] * sg) / s[:, None]
    sa = np.where(a >= 0, 1.0, -1.0)
    sb = np.where(b >= 0, 1.0, -1.0)
    lower = (v[:, 2] < 0)[:, None]
    dux = np.where(lower, -(sa * sb)[:, None] * db, da)
    duy = np.where(lower, -(sa * sb)[:, None] * da, db)
    return np.stack([dux, duy], axis=1)


def _barycentric_gradient(i0, j0, fx32, fy32, N):
    """d b_k / d(f_x, f_y) of vertex_triangle's weights: constant per
    triangle.  Returns [N][3][2]."""
    f = np.float32
    anti = (i0 >= N // 2) == (j0 >= N // 2)
    a_lower = (fx32 + fy32) <= f(1.0)
    m_lower = fy32 <= fx32
    g = np.zeros((len(i0), 3, 2))
    g[anti & a_lower] = [[-1, -1], [1, 0], [0, 1]]
    g[anti & ~a_lower] = [[1, 1], [0, -1], [-1, 0]]
    g[~anti & m_lower] = [[-1, 0], [1, -1], [0, 1]]
    g[~anti & ~m_lower] = [[0, -1], [-1, 1], [1, 0]]
    return g


def shifted_features_d_gradient(tree, tables, x, omega, normal, disparity):
    """dh/dd [N][K F] of encode_features_shifted: per level and cell j,
    sum_k wn_j (db_jk/dd) t_jk with db/dd = db/df (N/2) du/dv (x - c_j), the
    triangle and cells as the binary32 lookup decides them."""
    T = np.asarray(tables, dtype=np.float64)
    F = T.shape[1]
    n = len(x)
    K = tree.num_levels
    om_r = reflect_f32(omega, normal)
    x32 = np.clip(np.asarray(x, dtype=np.float32), np.float32(0), np.float32(1))
    enc = encode_features_shifted(tree, tables, x, omega, normal, disparity)
    out = np.zeros((n, K * F))
    for l in range(K):
        V = int(tree.R[l])
        N = V - 1
        cells, _, _ = neighbour_cells(x, l)
        for j in range(8):
            v = shifted_direction_f32(x, om_r, disparity, cells[:, j], l)
            i0, j0, fx32, fy32 = vertex_cell_f32(v, V)
            gb = _barycentric_gradient(i0, j0, fx32, fy32, N)          # [n][3][2]
            J = _fold_jacobian(v) * (N / 2.0)                          # d(px, py)/dv
            c = (cells[:, j] + 0.5) / 2.0 ** l
            dv = x32.astype(np.float64) - c                            # dv/dd
            dp = np.einsum("nab,nb->na", J, dv)                        # d(px, py)/dd
            dbk = np.einsum("nka,na->nk", gb, dp)                      # [n][3]
            # the cell's renormalised weight wn_j: its entries' weights
            # wn_j b_k summed over the triangle's vertices (sum_k b_k = 1)
            wcell = enc.weight[:, l, j, :].sum(axis=1)
            for k in range(3):
                a = enc.addr[:, l, j, k]
                ok = a >= 0
                out[ok, l * F:(l + 1) * F] += (wcell[ok] * dbk[ok, k])[:, None] * T[a[ok]]
    return out


def disparity_backward(table, res, weights, x, omega, normal, d_disp):
    """Gradients of sum_q d_disp[q] d_q (d = g_psi(x, omega_r)) with respect
    to the hash tables [L][T][2] and the MLP weights: dz = d_disp d (exp),
    the bias-free ReLU MLP's backward, and each level's feature gradient
    scattered to its cell's 8 vertices with the trilinear weights."""
    tab = np.asarray(table, dtype=np.float64)
    L, T, Fh = tab.shape
    om_r = reflect_f32(omega, normal).astype(np.float64)
    inp = np.concatenate([hash_encode(table, res, x), om_r], axis=1)
    out, zs, inputs = mlp_forward(weights, inp)
    Ws = [np.asarray(W, dtype=np.float64) for W in weights]
    delta = np.asarray(d_disp, dtype=np.float64)[:, None] * out
    dWs = [None] * len(Ws)
    for i in range(len(Ws) - 1, -1, -1):
        dWs[i] = delta.T @ inputs[i]
        g = delta @ Ws[i]
        if i > 0:
            delta = g * (zs[i - 1] > 0)
        else:
            d_in = g
    dtab = np.zeros_like(tab)
    x32 = np.clip(np.asarray(x, dtype=np.float32), np.float32(0), np.float32(1))
    for l in range(L):
        N = int(res[l])
        p = x32 * np.float32(N)
        i0 = np.minimum(np.floor(p), np.float32(N - 1)).astype(np.int64)
        f = p.astype(np.float64) - i0
        for c in range(8):
            dd = np.array([c & 1, (c >> 1) & 1, c >> 2])
            idx = hash_index(i0[:, 0] + dd[0], i0[:, 1] + dd[1], i0[:, 2] + dd[2], N, T)
            w = np.ones(len(x32))
            for a in range(3):
                w *= f[:, a] if dd[a] else 1.0 - f[:, a]
            for k in range(Fh):
                dtab[l, :, k] += np.bincount(idx, weights=w * d_in[:, l * Fh + k], minlength=T)
    return dtab, dWs


def disparity_gradient(tree, tables, weights, x, omega, normal, disparity, d_rgb, attrs=None):
    """d/dd_q of sum(d_rgb * L_hat) in the shifted form (Eq. 7-9) for every
    query q: the decoder's input gradient dh (Eq. 13 back-propagated, as in
    query_backward) dotted with the query's feature derivative dh/dd
    (shifted_features_d_gradient); the attributes of Eq. 12 do not depend
    on d.  The lookup takes d in binary32.  Returns [N] (FP64)."""
    d32 = np.asarray(disparity, dtype=np.float32)
    _, _, _, dh = query_backward(tree, tables, weights, x, omega, d_rgb, form="shifted",
                                 attrs=attrs, normal=normal, disparity=d32, return_dh=True)
    dhdd = shifted_features_d_gradient(tree, tables, x, omega, normal, d32)
    return np.sum(dh[:, :dhdd.shape[1]] * dhdd, axis=1)


def shifted_train_gradients(tree, tables, weights, predictor, pairs, normal, normal2, eps=1e-2,
                            rhs_grad=True, scale=1.0, attrs=None):
    """The gradients of one training step of the paper's full model, before
    the optimiser: every primary query (x, omega) and secondary query
    (x', -omega') predicts its disparity d = g_psi(x, omega_r) (Eq. 7; omega_r
    the reflection about that point's normal), reads the features with the
    disparity-shifted lookup (Eq. 8-9 with Eq. 6, 10; d rounded to binary32,
    the precision the lookup decides in) and is decoded (Eq. 13, with the
    attributes of Eq. 12 when given as [2N][n_attrs], primaries first);
    Eq. 14 against the one-sample target of Eq. 3 gives the loss.  The
    disparity is trained only through this objective (Section 3.3): each
    query's dL/dd (disparity_gradient) back-propagates through g_psi
    (disparity_backward).  predictor = (hash table [L][T][2], res, weights).
    Gradients are of scale * loss.  Returns (loss, dT, dWs, d_table, d_Ws_psi,
    dL/dd [2N], d [2N])."""
    table, res, pw = predictor
    n = len(pairs.x)
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    Nr = np.concatenate([normal, normal2])
    d = disparity(table, res, pw, X, Om, Nr)
    d32 = d.astype(np.float32)
    rgb, _ = query_forward(tree, tables, weights, X, Om, form="shifted", normal=Nr,
                           disparity=d32, attrs=attrs)
    loss, dLp, dLs = residual_loss(rgb[:n], rgb[n:], pairs.E, pairs.w, eps, rhs_grad, scale)
    d_rgb = np.concatenate([dLp, dLs])
    dT, dWs, _, dh = query_backward(tree, tables, weights, X, Om, d_rgb, form="shifted",
                                    attrs=attrs, normal=Nr, disparity=d32, return_dh=True)
    dhdd = shifted_features_d_gradient(tree, tables, X, Om, Nr, d32)
    dd = np.sum(dh[:, :dhdd.shape[1]] * dhdd, axis=1)
    dtab, dWp = disparity_backward(table, res, pw, X, Om, Nr, dd)
    return loss, dT, dWs, dtab, dWp, dd, d
