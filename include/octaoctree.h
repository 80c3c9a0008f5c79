/*
 * octaoctree.h -- C ABI of the GB300 (sm_103a) OctaOctree query and its
 * training step.
 *
 * The method (arxiv 2606.08469): outgoing radiance L(x, w) is read from a
 * multi-level sparse octree whose every non-empty cell stores an octahedral
 * feature map (Section 3.4).  A query finds, at every level, the node that
 * contains x, maps w onto the octahedral square (Section 3.3, Eq. 4 and
 * Eq. 5), blends the four surrounding texels of that node's map bilinearly,
 * concatenates the levels (Eq. 11) and decodes the features with a small MLP
 * (Section 3.5, Eq. 13).  Training minimises the relative-L2 residual between
 * the query and its emission-plus-secondary-query estimate (Eq. 3, Eq. 14).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an int status: OCTA_OK or a negative OCTA_E* code.
 *    No exception or abort crosses the ABI.  octa_last_error() returns a
 *    thread-local message for the last failing call on the calling thread.
 *  - Pointers documented as "device" are CUDA device pointers owned by the
 *    caller; the library never allocates, frees, synchronises or prints.
 *    GPU work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and runs asynchronously: results are valid once the stream
 *    reaches that point.
 *  - Pointers documented as "host" are read during the call only.
 *  - Scratch space comes from a caller-provided device workspace of at least
 *    octa_workspace_bytes(op, n) bytes, 256-byte aligned and zero-filled
 *    before its first use (every call leaves it ready for the next).  Two
 *    calls that share a workspace must not overlap on the GPU.
 *  - Device-detected malformed input (a child index or texel range outside
 *    the arrays) is never dereferenced: the level is treated as absent and
 *    the OCTA_STATUS_* bit is OR-ed into *status (device int32, nullable).
 */
#ifndef OCTAOCTREE_H
#define OCTAOCTREE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define OCTA_OK 0
#define OCTA_EINVAL (-1)      /* bad argument: NULL, shape, dtype, alignment  */
#define OCTA_ERANGE (-2)      /* size outside the supported range             */
#define OCTA_ECUDA (-3)       /* CUDA launch error; text in octa_last_error() */
#define OCTA_ETIMEOUT (-4)    /* a bounded device wait gave up                */
#define OCTA_EUNSUPPORTED (-6)/* valid but not built (e.g. a width/dtype mix) */

/* bits OR-ed into the device status word */
#define OCTA_STATUS_BAD_CHILD 1   /* first_child[n] + 7 >= num_nodes          */
#define OCTA_STATUS_BAD_MAP 2     /* map_offset[n] + R^2 > num_texels         */
#define OCTA_STATUS_TIMEOUT 4     /* bounded grid barrier gave up             */

/* ---- limits ------------------------------------------------------------ */
#define OCTA_MAX_LEVELS 16
#define OCTA_MAX_LAYERS 6         /* weight matrices per MLP                  */
#define OCTA_MAX_SCENES 16
#define OCTA_MAX_GROUPS 16        /* Adam parameter groups per call           */

/* ---- element types ----------------------------------------------------- */
#define OCTA_F32 0
#define OCTA_F16 1
#define OCTA_BF16 2

/* ---- octree ------------------------------------------------------------ */
/* Level-ordered flat octree.  Level l holds nodes
 * [level_node_start[l], level_node_start[l+1]); the 8 children of node n are
 * first_child[n] + b, b = bx | by<<1 | bz<<2 (Morton order), or
 * first_child[n] = -1 for a leaf.  Node n of level l owns the R[l] x R[l]
 * texels starting at map_offset[n]; texel (i, j) of that map (i along u_x)
 * is texel index map_offset[n] + j*R[l] + i of the feature table
 * [num_texels][F].  level_texel_base[l] is the first texel of level l.   */
typedef struct octa_tree_desc {
  int32_t num_levels;                          /* K = max_depth + 1        */
  int32_t num_nodes;
  int64_t num_texels;
  int32_t R[OCTA_MAX_LEVELS];                  /* map side per level       */
  int32_t level_node_start[OCTA_MAX_LEVELS + 1];
  int64_t level_texel_base[OCTA_MAX_LEVELS + 1];
} octa_tree_desc;

/* octree_build -- seeded adaptive octree over [0,1]^3 (host only).
 * Nodes are created breadth first.  A node at depth d < max_depth draws one
 * SplitMix64 uniform u (Steele et al. 2014; state seeded with `seed`, one
 * draw per such node in node order, u = (z >> 11) * 2^-53) and splits into 8
 * children iff u < p_base^d (p_base^d = product of d factors, from 1.0).
 * The paper builds its octree from the scene geometry (Section 3.4, Section
 * 4.1); this seeded generator stands in for it.
 * Two-call sizing: with first_child == NULL only *desc is filled; then call
 * again with caller-owned host arrays first_child[num_nodes],
 * node_coord[num_nodes][3] (integer cell coordinates at the node's level)
 * and map_offset[num_nodes].
 * R: host [max_depth+1], each 2..4096.  max_depth 0..OCTA_MAX_LEVELS-1.
 * Errors: OCTA_EINVAL (NULL desc/R, p_base outside [0,1]), OCTA_ERANGE
 * (depth, R, more than 2^31-1 nodes or texels).                            */
int octree_build(uint64_t seed, int32_t max_depth, double p_base, const int32_t* R,
                 octa_tree_desc* desc, int32_t* first_child, int32_t* node_coord,
                 int32_t* map_offset);

/* octree_from_flags -- same output for a hand-written tree: the k-th node (in
 * breadth-first order) whose depth is below max_depth splits iff
 * k < n_flags && flags[k] != 0.  flags: host, may be NULL when n_flags == 0.*/
int octree_from_flags(const uint8_t* flags, int64_t n_flags, int32_t max_depth,
                      const int32_t* R, octa_tree_desc* desc, int32_t* first_child,
                      int32_t* node_coord, int32_t* map_offset);

/* ---- scene: one octree, its feature table and its decoder -------------- */
typedef struct octa_scene {
  const int32_t* first_child;  /* device [num_nodes]                       */
  const int32_t* map_offset;   /* device [num_nodes]                       */
  const void* tables;          /* device [num_texels][F], table_dtype      */
  const void* weights;         /* device: W_1..W_L back to back, each      */
                               /* row-major [widths[i+1]][widths[i]]       */
  int32_t num_levels;          /* K (1..OCTA_MAX_LEVELS)                   */
  int32_t num_nodes;
  int64_t num_texels;          /* < 2^31                                   */
  int32_t R[OCTA_MAX_LEVELS];  /* map side per level (2..4096)             */
  int32_t F;                   /* features per texel: 4 or 8               */
  int32_t table_dtype;         /* OCTA_F32 or OCTA_F16                     */
  int32_t weight_dtype;        /* OCTA_F32 or OCTA_BF16                    */
  int32_t n_layers;            /* weight matrices L (2..OCTA_MAX_LAYERS)   */
  int32_t widths[OCTA_MAX_LAYERS + 1]; /* widths[0] = K*F, widths[L] = 3   */
  int32_t query_form;          /* OCTA_FORM_CELL_BILINEAR or
                                  OCTA_FORM_TRILINEAR_VERTEX (see below)   */
} octa_scene;

/* Query forms.  OCTA_FORM_CELL_BILINEAR: per level the cell that contains x
 * and a bilinear blend of the 4 texels around the direction on its R x R
 * texel-centred map.  OCTA_FORM_TRILINEAR_VERTEX (Eq. 10 with Eq. 6, without
 * the disparity shift): per level the 8 cells around x with trilinear
 * weights renormalised over the cells present in the octree, in each the
 * barycentric blend of the 3 vertices of the triangle holding the direction
 * on the node's R x R vertex map (R = 2^k + 1, k >= 1; mirrored vertices of
 * the map's edges are one vertex).  Every query and training entry point
 * evaluates either form, for FP32 and BF16 decoders.                      */
#define OCTA_FORM_CELL_BILINEAR 0
#define OCTA_FORM_TRILINEAR_VERTEX 1
/* OCTA_FORM_SHIFTED (Eq. 7-9 with Eq. 10 and Eq. 6): the trilinear vertex
 * form in which cell j of a level looks its map up in the direction of
 * y - c_j, y = x + omega_r / d (c_j the cell's centre, d the query's
 * disparity, omega_r the reflection of omega about the normal, both
 * normalised as v / sqrt(v.v)), evaluated as (x - c_j) d + omega_r in
 * binary32 with one rounding per operation (omega_r = (2 (n.omega)) n -
 * omega; the octahedral map divides by the L1 norm, so no normalisation).
 * octa_encode, octa_query_fwd, octa_query_bwd and octa_train_fused
 * evaluate it (FP32 decoders: F = 8; octa_train_step_batched returns
 * OCTA_EUNSUPPORTED); the disparity comes from the caller (octa_disparity
 * computes it with the predictor g_psi).  The backward passes can also
 * return each query's dL/dd (d_disparity), the derivative through every
 * cell's shifted direction, the octahedral fold and the triangle's
 * barycentric weights; octa_disparity_bwd carries it into g_psi, which
 * the paper trains only through the radiance objective (Section 3.3).    */
#define OCTA_FORM_SHIFTED 2

/* Queries: scene s answers queries [scene_start[s], scene_start[s+1]).   */
typedef struct octa_queries {
  const float* x;              /* device [n][3], position (clamped to [0,1])*/
  const float* omega;          /* device [n][3], direction (any length > 0) */
  int64_t n;
  int64_t scene_start[OCTA_MAX_SCENES + 1];
  /* the shifted form only (NULL otherwise): */
  const float* normal;         /* device [n][3], surface normal (length > 0)*/
  const float* disparity;      /* device [n], d of Eq. 8 (>= 0)            */
  /* Eq. 12's surface attributes g, appended to the decoder input after the
   * K*F features (widths[0] = K*F + n_attrs); the paper's g is position,
   * reflection direction, normal, albedo and roughness (13 values).  Read
   * by octa_query_fwd and octa_query_bwd; NULL / 0 for none.              */
  const float* attrs;          /* device [n][n_attrs]                       */
  int32_t n_attrs;             /* 0..OCTA_MAX_ATTRS                         */
  int32_t reserved_q;
  /* octa_query_bwd in the shifted form: written with dL/dd of every query,
   * the gradient (of the same loss as the table and weight gradients)
   * with respect to its disparity; NULL: not computed.                    */
  float* d_disparity;          /* device [n]                                */
} octa_queries;
#define OCTA_MAX_ATTRS 16

/* octa_encode -- the OctaOctree encoding alone in the scenes' query form
 * (all scenes of a call share it; Eq. 10 single-cell bilinear form, Eq. 10
 * with Eq. 6, or the shifted form of Eq. 7-9 with q->normal and
 * q->disparity; then Eq. 11): each query writes its own scene's K*F features
 * into a row of row_stride elements (row_stride >= K*F of every scene;
 * unused tail left untouched).  feat_dtype OCTA_F32 or OCTA_BF16.  Absent
 * levels write zeros.  node_idx: device [n][K_max] int32 or NULL (K_max =
 * largest K of the scenes, unused columns -1; cell form only).
 * texel_addr: device int32 or NULL, -1 where absent: cell form [n][K_max][4]
 * (corner k = a + 2b for corner (i0+a, j0+b)); trilinear vertex and
 * shifted forms [n][K_max][24] (neighbour j = 0..7, offset (j & 1, j >> 1 & 1, j >> 2)
 * from the lower cell, times vertex k = 0..2: entry 3 j + k).             */
int octa_encode(const octa_scene* scenes, int32_t n_scenes, const octa_queries* q,
                void* features, int32_t feat_dtype, int64_t row_stride,
                int32_t* node_idx, int32_t* texel_addr, int32_t* status, void* stream);

/* octa_query_fwd -- L_hat(x, omega) = exp(W_L relu(... relu(W_1 h))) per
 * query (Eq. 13), h the encoding above.  rgb: device [n][3] float32.
 * node_idx / texel_addr / status as in octa_encode (nullable; the scenes
 * of a call share one query form, node_idx only in the cell form).
 * The FP32 path (weight_dtype F32) runs on the CUDA cores in FP32; the
 * BF16 path runs the decoder on the tcgen05 tensor cores (BF16 operands,
 * FP32 accumulation in tensor memory).                                     */
int octa_query_fwd(const octa_scene* scenes, int32_t n_scenes, const octa_queries* q,
                   float* rgb, int32_t* node_idx, int32_t* texel_addr, int32_t* status,
                   void* stream);

/* Gradient buffers of one scene: FP32, same layouts as tables / weights.  */
typedef struct octa_scene_grads {
  float* d_tables;             /* device [num_texels][F], 16-byte aligned  */
  float* d_weights;            /* device, layout of octa_scene.weights     */
} octa_scene_grads;

/* octa_query_bwd -- gradients of sum_q d_rgb[q] . L_hat(q) with respect to
 * the feature tables and the decoder weights.  Recomputes the forward pass
 * (no activations are kept between calls), back-propagates through the
 * decoder (exp, ReLU masks 1[z > 0]) and scatter-adds weight_k * dh_l into
 * the entries each present level read (4 texels in the cell form; in the
 * trilinear vertex form 24 vertices, weight = renormalised cell weight x
 * barycentric weight).  ACCUMULATES (+=) into
 * grads[s].d_tables / d_weights, which the caller zeroes (adam_step zeroes
 * them after each update).  d_rgb: device [n][3] float32.                 */
int octa_query_bwd(const octa_scene* scenes, int32_t n_scenes, const octa_queries* q,
                   const float* d_rgb, const octa_scene_grads* grads, int32_t* status,
                   void* stream);

/* ---- loss scaler / optimiser state (device resident) ------------------- */
typedef struct octa_scaler {
  float scale;                 /* current loss scale S                     */
  float inv_scale_used;        /* 1/S applied to the last step's gradients */
  int32_t good_steps;          /* consecutive finite steps since a change  */
  int32_t growth_interval;     /* double S after this many finite steps;   */
                               /* 0 = static scale                         */
  int32_t step;                /* Adam step count t of applied steps       */
  int32_t skipped;             /* 1 if the last step was skipped           */
  int32_t n_skipped;           /* total skipped steps                      */
  int32_t reserved;
  double grad_norm;            /* ||g / S||_2 of the last step (FP64)      */
  double loss;                 /* free slot for residual_loss's output     */
} octa_scaler;

/* residual_loss -- Eq. 14 with the one-sample target of Eq. 3:
 * T = E + w * L_s,  r = (L_p - T) / (L_p + T + eps),
 * loss = sum(r^2) / (3 n_pairs)  (FP64 reduction, deterministic),
 * dL_p = S * 2 r / (3 n (L_p + T + eps)), and, if rhs_grad,
 * dL_s = -S * 2 r w / (3 n (L_p + T + eps)) (gradient through the target's
 * secondary query; the normaliser stays detached).  S = scaler->scale or 1
 * when scaler is NULL.  All arrays device [n_pairs][3] float32; dL_s may be
 * NULL when rhs_grad == 0 (else it is written with zeros).
 * loss_dev: device double.  Workspace: octa_workspace_bytes(OCTA_OP_LOSS, n).*/
int residual_loss(const float* L_p, const float* L_s, const float* E, const float* w,
                  int64_t n_pairs, float eps, int32_t rhs_grad, const octa_scaler* scaler,
                  double* loss_dev, float* dL_p, float* dL_s, void* workspace,
                  size_t workspace_bytes, void* stream);

/* residual_loss_static -- residual_loss without a workspace argument.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory -- for example code in a renderer's per-frame path,
 * where a cudaMalloc may synchronise the device and stall the frame, or a
 * plug-in whose host application owns every device allocation.  The scratch
 * (per-block FP64 partials and a completion counter) lives in a fixed
 * 16.6 KB array inside the library that every GPU which loads it keeps until
 * the process exits.  The call allocates nothing and calls no allocating
 * routine.  Limits: n_pairs <= 2,796,202 (the partial slots of the fixed
 * array); larger batches return OCTA_ERANGE with a message -- use
 * residual_loss with a workspace for them.  The current device's index must
 * be below 64 (the library keeps the array's address for devices 0..63);
 * a higher index returns OCTA_ERANGE.  The first call on a device looks
 * the array's device address up (cudaGetSymbolAddress) for that device, so
 * make that first call before any stream capture.  Every call shares the one
 * array: each call clears its counter on `stream` before the kernel, and
 * calls that overlap on the GPU (other streams, other threads) race and give
 * wrong losses.  Arguments, outputs and gradients are those of
 * residual_loss; the loss is summed in another block order, so it agrees
 * with residual_loss to FP64 rounding, the gradients exactly.             */
int residual_loss_static(const float* L_p, const float* L_s, const float* E, const float* w,
                         int64_t n_pairs, float eps, int32_t rhs_grad,
                         const octa_scaler* scaler, double* loss_dev, float* dL_p, float* dL_s,
                         void* stream);

/* ---- the disparity predictor g_psi (Eq. 7, Section 3.5) ---------------- */

/* g_psi: a multiresolution hash encoding of x -- level l's grid has res[l]
 * cells a side; p = x res[l] in binary32 (x clamped to [0,1]), cell
 * i0 = min(floor(p), res[l] - 1) per axis, trilinear weights of p - i0;
 * vertex (i, j, k) is entry i + j (N+1) + k (N+1)^2 of the level's table
 * when (N+1)^3 <= T, else (i * 1 ^ j * 2654435761 ^ k * 805459861) mod T in
 * 32-bit unsigned arithmetic (Mueller et al. 2022) -- concatenated with
 * omega_r (the reflection of omega about the normal, as in the shifted
 * form), into a bias-free MLP (2 levels + 3) -> 64 -> 64 -> 1 with ReLU
 * hidden layers and an exp output, so the disparity d is positive.       */
#define OCTA_PRED_HIDDEN 64
#define OCTA_PRED_MAX_LEVELS 16
typedef struct octa_predictor {
  const float* table;          /* device [levels][2^log2_T][2] float32     */
  const float* weights;        /* device W1 [64][2 levels + 3], W2 [64][64],*/
                               /* W3 [1][64], row-major, back to back      */
  const void* weights_bf16;    /* NULL: the MLP runs in FP32 on the CUDA
                                  cores; else the same weights in BF16 and
                                  the MLP runs on the tcgen05 tensor cores
                                  (BF16 operands, FP32 accumulation; levels
                                  <= 14)                                  */
  int32_t levels;              /* 1..OCTA_PRED_MAX_LEVELS                  */
  int32_t log2_T;              /* 4..24                                    */
  int32_t res[OCTA_PRED_MAX_LEVELS]; /* cells a side per level, 1..65535  */
} octa_predictor;

/* octa_disparity -- d = g_psi(x, omega_r) for queries q (x, omega and
 * normal; scene_start is not used).  disparity: device [n] float32, the
 * shifted form's input.                                                   */
int octa_disparity(const octa_predictor* pred, const octa_queries* q, float* disparity,
                   void* stream);

/* octa_disparity_bwd -- g_psi's backward (Section 3.3: d is trained through
 * the radiance objective alone): the gradients of sum_q d_disp[q] d_q with
 * respect to the hash tables and the MLP weights.  Recomputes the forward,
 * back-propagates through exp (dd/dz = d) and the ReLU layers, and scatter-
 * adds each level's two feature gradients into its cell's eight vertices
 * with the trilinear weights (float2 atomics).  With pred->weights_bf16 NULL
 * everything runs in FP32 on the CUDA cores (pred->weights); otherwise the
 * MLP's forward and backward run on the tcgen05 tensor cores from the BF16
 * weights (BF16 operands, FP32 accumulation; levels <= 14), as octa_disparity
 * does.  ACCUMULATES (+=) into d_table
 * (device float32, layout of pred->table, 8-byte aligned) and d_weights
 * (device float32, layout of pred->weights), which the caller zeroes.
 * d_disp: device [n] float32 (the shifted backward's d_disparity).        */
int octa_disparity_bwd(const octa_predictor* pred, const octa_queries* q, const float* d_disp,
                       float* d_table, float* d_weights, void* stream);

/* ---- the training regime of Section 4: M RHS samples per LHS sample ---- */

/* residual_loss_multi -- Eq. 14 against Eq. 3's M-sample target:
 * T = E + (1/M) sum_m w_m * L_s,m  (M = n_samples >= 1),
 * r = (L_p - T) / (L_p + T + eps), loss = sum(r^2) / (3 n_pairs) (FP64
 * reduction, deterministic for a given launch shape),
 * dL_p = S * 2 r / (3 n (L_p + T + eps)) and, if rhs_grad,
 * dL_s,m = -dL_p * w_m / M (the gradient through the target into every
 * secondary radiance; the normaliser stays detached).  Without rhs_grad the
 * target is detached as Eq. 14 prints and dL_s (nullable) gets zeros.
 * S = scaler->scale or 1 when scaler is NULL.  L_p, E, dL_p: device
 * [n_pairs][3] float32; L_s, w, dL_s: device [n_pairs][M][3] float32 (the M
 * samples of a pair contiguous).  loss_dev: device double.  Workspace:
 * octa_workspace_bytes(OCTA_OP_LOSS, n_pairs).  M = 1 gives residual_loss's
 * values (the loss to FP64 rounding).                                     */
int residual_loss_multi(const float* L_p, const float* L_s, const float* E, const float* w,
                        int64_t n_pairs, int32_t n_samples, float eps, int32_t rhs_grad,
                        const octa_scaler* scaler, double* loss_dev, float* dL_p, float* dL_s,
                        void* workspace, size_t workspace_bytes, void* stream);

/* The synthetic scene that secondary rays hit (Eq. 2): planes (square
 * patches |(x - p).t1| <= h, |(x - p).t2| <= h, or unbounded with h = inf),
 * spheres, and always the six inner walls of the unit box.              */
#define OCTA_MAX_PRIMS 64
typedef struct octa_prims {
  const float* planes;         /* device [n_planes][13]: point p(3), unit    */
                               /* normal n(3), tangents t1(3), t2(3), h     */
  const float* spheres;        /* device [n_spheres][4]: centre(3), radius  */
  int32_t n_planes;            /* 0..OCTA_MAX_PRIMS                         */
  int32_t n_spheres;           /* 0..OCTA_MAX_PRIMS                         */
} octa_prims;

/* octa_trace_rays -- x'(omega_i) of Eq. 2: the first intersection with t >
 * t_min of ray i, origin[i / rays_per_origin] + t dir[i], with the scene.
 * Every decision is taken in binary32 with one rounding per operation in a
 * fixed order (plane: t = ((p - o).n) / (d.n), hit on the patch; sphere
 * with |d| = 1: b = (o - c).d, disc = b^2 - ((o - c).(o - c) - r^2),
 * t = -b - sqrt(disc) if that exceeds t_min, else -b + sqrt(disc); wall
 * a at w: t = (w - o_a) / d_a; dot products ((x0 y0 + x1 y1) + x2 y2);
 * planes, spheres, then walls x0, x1, y0, y1, z0, z1, each replacing the
 * best hit only on a strictly smaller t), so results are bit-reproducible.
 * Outputs (device, n_rays rows): hit [n][3] = o + t d per component
 * (required); query_dir [n][3] = -dir, the secondary query's direction
 * (nullable); prim [n] int32 = planes 0..P-1, spheres P..P+S-1, walls
 * P+S+2a+(w == 1), -1 for a miss (nullable); t [n] (nullable, inf for a
 * miss).  origin / dir: device float32 [.][3].  rays_per_origin >= 1.     */
int octa_trace_rays(const octa_prims* prims, const float* origin, int32_t rays_per_origin,
                    const float* dir, int64_t n_rays, float t_min, float* hit,
                    float* query_dir, int32_t* prim, float* t, void* stream);

/* Training pairs: pair i of scene s (scene_start[s] <= i < scene_start[s+1])
 * is the primary query (x[i], omega[i]) and the secondary query
 * (x2[i], omega2[i]); omega2 is the secondary query's direction itself,
 * i.e. -omega' for a sampled incident direction omega' (Eq. 2).          */
typedef struct octa_pairs {
  const float* x;              /* device [n][3] primary positions           */
  const float* omega;          /* device [n][3] primary outgoing directions */
  const float* x2;             /* device [n][3] secondary positions x'      */
  const float* omega2;         /* device [n][3] secondary query directions  */
  const float* E;              /* device [n][3] emitted radiance at x       */
  const float* w;              /* device [n][3] f_r |n.omega'| / p(omega')  */
  int64_t n;
  int64_t scene_start[OCTA_MAX_SCENES + 1];
  /* pairs that scene s's loss is a mean over (0: its own count).  A data-
   * parallel rank holding a shard of a batch passes the whole batch's count,
   * so that its loss and gradients are its shard's share of the batch's and
   * the ranks' sums are the batch's.                                        */
  int64_t norm_pairs[OCTA_MAX_SCENES];
  /* the shifted form only (NULL otherwise): the primary and secondary
   * queries' normals [n][3] and disparities [n], and (nullable) outputs
   * d_disparity / d_disparity2 [n] written with each query's dL/dd (the
   * gradient of S * loss, as the table and weight gradients).             */
  const float* normal;
  const float* normal2;
  const float* disparity;
  const float* disparity2;
  float* d_disparity;
  float* d_disparity2;
} octa_pairs;

/* octa_train_fused -- octa_query_fwd + residual_loss + octa_query_bwd of a
 * training batch in one launch: BF16 decoders on the tensor cores, FP32
 * decoders on the FP32 engine (CUDA cores); all scenes share the dtype.
 * Every 64-pair tile runs the primary and secondary queries together, forms
 * the Eq. 14 gradient of each pair from its two radiances in the tile
 * (the target's dependence on the secondary query enters iff rhs_grad; the
 * normaliser is detached), and back-propagates into the tables and the
 * decoder (gradients of S * loss, S = scaler->scale or 1; accumulated into
 * grads as in octa_query_bwd).  loss_dev: device double [n_scenes], set to
 * each scene's sum of r^2 over its pairs and channels divided by 3 x
 * (pairs->norm_pairs[s], or the scene's own pair count when 0) (zeroed by
 * the call; FP64 partials, summed with atomics); the gradients are of that
 * same loss.  OCTA_EUNSUPPORTED for scenes of mixed decoder dtypes;
 * OCTA_EINVAL for a negative norm_pairs.                                  */
int octa_train_fused(const octa_scene* scenes, int32_t n_scenes, const octa_pairs* pairs,
                     float eps, int32_t rhs_grad, const octa_scaler* scaler, double* loss_dev,
                     const octa_scene_grads* grads, int32_t* status, void* stream);

/* One parameter group of adam_step (all device pointers, n elements).     */
typedef struct octa_param_group {
  float* param;                /* FP32 master copy                          */
  float* grad;                 /* FP32 gradient of S * loss; zeroed after   */
  float* m;                    /* first moment                              */
  float* v;                    /* second moment                             */
  void* work;                  /* low-precision working copy or NULL        */
  int32_t work_dtype;          /* OCTA_F16 or OCTA_BF16                     */
  float lr;
  int64_t n;
} octa_param_group;

typedef struct octa_adam_cfg {
  float beta1, beta2, eps;     /* Kingma & Ba defaults 0.9, 0.999, 1e-8     */
} octa_adam_cfg;

/* adam_step -- unscale by 1/S, FP64 gradient norm and non-finite check,
 * then either skip the step and halve S (non-finite; scaler->skipped = 1) or
 * apply Adam with bias correction at t = ++scaler->step and, after
 * growth_interval consecutive finite steps, double S (Micikevicius et al.
 * 2018).  Writes the working copies, zeroes every grad.  All decisions are
 * taken on the device (no host sync).  scaler: device, initialised by the
 * caller.  Workspace: octa_workspace_bytes(OCTA_OP_ADAM, total elements).  */
int adam_step(const octa_param_group* groups, int32_t n_groups, const octa_adam_cfg* cfg,
              octa_scaler* scaler, void* workspace, size_t workspace_bytes, void* stream);

/* Options of octa_train_step_batched (nullable: defaults).                */
typedef struct octa_step_options {
  uint64_t barrier_timeout_ns; /* bound of each grid-barrier wait; 0 = 1 s  */
  int32_t extra_barrier_arrivals; /* test hook: arrivals the barriers await
                                  beyond the grid (0 in use; > 0 makes every
                                  wait run out, report OCTA_STATUS_TIMEOUT and
                                  skip the optimiser)                        */
  int32_t skip_first_mma;      /* test hook (0 in use): nonzero = no CTA
                                  issues the tensor-core MMAs of the first
                                  layer of its first tile, so that group's
                                  mbarrier wait (bounded by
                                  barrier_timeout_ns, like the grid barriers)
                                  runs out: the kernel reports
                                  OCTA_STATUS_TIMEOUT, frees its tensor
                                  memory and returns without the optimiser */
} octa_step_options;

/* octa_train_step_batched -- a whole training step of up to 16 scenes in one
 * persistent cooperative launch: the fused pass of octa_train_fused over all
 * pairs, then (after a grid-wide barrier) the FP64 gradient norm from
 * per-CTA partials, the loss-scale decision and Adam over the parameter
 * groups (after a second barrier), exactly as adam_step.  grads[s] must
 * alias the grad buffers of the groups that hold scene s's parameters and
 * start zeroed (every step leaves them zeroed).  Every barrier wait is
 * bounded; on timeout OCTA_STATUS_TIMEOUT is set in *status and the step is
 * incomplete; the call clears the barrier words of the workspace on `stream`
 * before its launch, so the next call starts from a consistent state.
 * Workspace: octa_workspace_bytes(OCTA_OP_STEP, 0).  BF16 decoders only.  */
int octa_train_step_batched(const octa_scene* scenes, int32_t n_scenes, const octa_pairs* pairs,
                            const octa_scene_grads* grads, const octa_param_group* groups,
                            int32_t n_groups, float eps, int32_t rhs_grad,
                            const octa_adam_cfg* adam, octa_scaler* scaler, double* loss_dev,
                            const octa_step_options* options, void* workspace,
                            size_t workspace_bytes, int32_t* status, void* stream);

/* ---- launch tuning ------------------------------------------------------ */
/* Process-wide launch knobs read by later calls (an autotuner sets them).
 * Zero in a field keeps the library's default.                            */
typedef struct octa_tuning {
  int32_t fwd_ctas_per_sm;     /* tensor-core forward: cap on resident CTAs
                                  per SM (each CTA = one 128-query tile)   */
  int32_t encode_ctas_per_sm;  /* octa_encode: cap on resident CTAs per SM */
  int32_t engine_ctas_per_sm;  /* FP32 path: cap on resident CTAs per SM   */
  int32_t fwd_order;           /* forward / encode / FP32 tiles: 1 = each
                                  persistent CTA takes a contiguous chunk,
                                  2 = interleaved (default)                */
  int32_t train_order;         /* training / backward work items: as above */
  int32_t fwd_threads_per_query; /* tensor-core forward: 1 (default) or 2
                                  threads per query (256-thread CTAs, each
                                  thread gathering half of the levels)     */
  int32_t encode_threads_per_query; /* octa_encode, cell form: 1 (default)
                                  or 2, as fwd_threads_per_query           */
  int32_t train_threads_per_row; /* tensor-core backward / training kernels,
                                  cell form: 2 (default: 512-thread CTAs,
                                  the two threads of a tile row splitting
                                  its levels and epilogue columns) or 1   */
  int32_t fwd_run;             /* queries per CTA work unit, in tiles of 128
                                  queries: with the interleaved order a
                                  persistent CTA of the forward, encoding
                                  and FP32 forward kernels takes fwd_run
                                  consecutive tiles at a time (1..64;
                                  default 1)                               */
  int32_t train_run;           /* the same for the backward and training
                                  kernels (work units: tensor-core items of
                                  two 128-row tiles, FP32 tiles)           */
  int32_t gather_stages;       /* cell-form gathers of 16-byte texels at one
                                  thread per query (octa_encode): 1 (default)
                                  = the texel loads land in registers, two
                                  levels in flight; 2..4 = they land in a shared-
                                  memory ring (cp.async) of that many
                                  levels, all in flight (8 KB of shared
                                  memory per level and 128-query CTA)      */
  int32_t l1_carveout;         /* shared-memory carveout of the gather,
                                  forward and FP32 kernels: 1 = the largest
                                  (least L1 cache), 2 (default) = the smallest that
                                  holds their resident CTAs, the rest of
                                  the SM's L1 / shared array caching the
                                  texel loads.  The one-launch training
                                  step always takes the largest.           */
} octa_tuning;
int octa_set_tuning(const octa_tuning* t);   /* NULL restores the defaults */
int octa_get_tuning(octa_tuning* t);

/* ---- workspace sizing, errors ------------------------------------------ */
#define OCTA_OP_LOSS 1
#define OCTA_OP_ADAM 2
#define OCTA_OP_STEP 3
size_t octa_workspace_bytes(int32_t op, int64_t n);

const char* octa_last_error(void);
int32_t octa_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OCTAOCTREE_H */
