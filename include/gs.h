/*
 * gs.h -- C ABI of the GB300 (sm_103a) semantic Gaussian-splatting rasterizer.
 *
 * The library implements the data-parallel hot path of ActiveSGM's mapping
 * backbone (arXiv 2506.00225): tile-based differentiable rasterization of
 * anisotropic 3D Gaussians with colour, depth, silhouette (Sec. 3.1, Eq. 1)
 * and the sparse top-k semantic distribution (Sec. 3.1, Eq. 3), its adjoint,
 * and batched candidate-view rendering of the exploration criteria
 * (Sec. 3.2, Eq. 6 and Eq. 7 with Eq. 4).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - All array arguments are DEVICE pointers owned by the caller, except the
 *   structs themselves (host memory, read during the call only) and the
 *   explicit host buffers of gs_read_counters / gs_status_string.
 * - The library allocates nothing.  Scratch memory is a caller-allocated
 *   device workspace of gs_workspace_size() bytes (256-byte aligned); it
 *   carries state from gs_project to gs_bin_sort to gs_render_fwd to
 *   gs_render_bwd, so these calls must receive the same scene sizes, cameras,
 *   config and workspace.
 * - Every call is asynchronous and stream-ordered on `stream` (a
 *   cudaStream_t; NULL = legacy default stream).  No call synchronises the
 *   host except gs_read_counters.  No call reads data-dependent sizes back to
 *   the host, so a chain of calls can be captured in a CUDA graph.
 * - Host-detectable argument errors return GS_ERR_ARG before anything is
 *   enqueued.  Launch failures return GS_ERR_CUDA.  Data-dependent device
 *   errors (more visible Gaussians or more (tile, Gaussian) pairs than the
 *   workspace holds) set a sticky status word in the workspace; later kernels
 *   of the chain skip their work and gs_read_counters reports it.  Nothing
 *   traps.
 * - Floating point is IEEE FP32.  Projection and binning use no fused
 *   multiply-add, so tile lists are reproducible bit for bit.
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same handle as cudaStream_t. */
typedef struct CUstream_st *gs_stream_t;

typedef enum gs_status {
  GS_OK = 0,
  GS_ERR_ARG = 1,         /* invalid argument (host check) */
  GS_ERR_CAPACITY = 2,    /* workspace capacity exceeded (device status) */
  GS_ERR_CUDA = 3,        /* CUDA launch or runtime error */
  GS_ERR_TIMEOUT = 4,     /* a bounded device wait gave up (device status) */
  GS_ERR_UNSUPPORTED = 5, /* configuration not compiled in */
  GS_ERR_TOO_LARGE = 6    /* sizes need more scratch than gs_render_fwd_noalloc has */
} gs_status;

/* Gaussian map, structure of arrays (Sec. 3.1 "Gaussian Mapping" and
 * "Sparse Semantic Representation").  n Gaussians, top-k semantics over m
 * classes (m includes the "unknown" class).
 *   means   [n,3]  world position (metres)
 *   scales  [n,3]  linear axis scales (already exponentiated)
 *   quats   [n,4]  rotation (w,x,y,z); normalised inside, need not be unit
 *   opacity [n]    in (0,1) (already through the sigmoid)
 *   rgb     [n,3]  view-independent colour
 *   sem_ids [n,k]  class ids in [0,m), fixed after initialisation
 *   sem_w   [n,k]  class probabilities (blended as given, not renormalised)
 *   geo_unc [n]    per-Gaussian scalar uncertainty, or NULL (candidates only)
 * Limits: 1 <= k <= 16, 1 <= m <= 1024, 0 <= n < 2^28. */
typedef struct gs_scene {
  int32_t n, k, m;
  const float *means, *scales, *quats, *opacity, *rgb;
  const int32_t *sem_ids;
  const float *sem_w;
  const float *geo_unc;
} gs_scene;

/* Pinhole camera, OpenCV axes (x right, y down, z forward).  w2c is the
 * row-major 3x4 world-to-camera [R | t].  Pixel (x, y) has centre
 * (x + 0.5, y + 0.5).  Limits: 1 <= width, height <= 16384, near > 0. */
typedef struct gs_camera {
  int32_t width, height;
  float fx, fy, cx, cy;
  float near_plane;
  float w2c[12];
} gs_camera;

/* Launch configuration.
 *   tile_w, tile_h       screen tile (compiled shapes: 16x16, 16x8, 8x8, 32x8)
 *   px_per_thread        pixels per thread in the adjoint: 1, 2 or 4 (4: 16x16
 *                        tiles only)
 *                        (0 = default 2); results do not depend on it
 *   sem_detach_geometry  1 (default in the Python layer): the semantic
 *                        upstream gradient reaches sem_w only, never the
 *                        geometric attributes (Sec. 3.1 "Semantic Loss",
 *                        last paragraph; Sec. 6 "Limited Joint Optimization")
 *   record_capacity      max visible (view, Gaussian) records in the
 *                        workspace; <= 0 means n * n_views (never overflows)
 *   pair_capacity        max (tile, Gaussian) pairs; <= 0 means
 *                        8 * record_capacity
 *   recompute_bwd        0: the forward keeps one bit per (pixel, staged
 *                        Gaussian) that contributed (pair_capacity / 8 bytes
 *                        per tile pixel), read by the semantic pass and the
 *                        adjoint; 1: no per-pixel storage besides the final
 *                        transmittance and last contributor -- both re-test
 *                        every (pixel, Gaussian) pair of the tile instead.
 *                        Results are identical.
 *   spin_limit           bound on the polls of one inter-CTA wait (decoupled
 *                        look-back of the sorts and of the single-view
 *                        projection); 0 = default (about 4
 *                        million polls with a short sleep each).  A wait that
 *                        runs out raises GS_ERR_TIMEOUT in the device status,
 *                        later kernels of the chain skip their work, and
 *                        gs_read_counters reports it.  Small values exist to
 *                        exercise that path.
 *   cand_bits_bytes      candidate renders (n_views > 1): bytes of contributor
 *                        bits the workspace keeps (0 = 4 GiB).  The views are
 *                        rendered in waves whose bits fit; a tile whose bits
 *                        still do not fit re-tests its pairs.  Results do not
 *                        depend on it.
 *   cand_batch           Gaussians staged per batch in the candidate kernels:
 *                        32, 64 or 128 (0 = 64); results do not depend on it
 *   cand_group_pixels    0 (default): gs_render_candidates projects, bins
 *                        and renders all its views at once.  P > 0: it does
 *                        so for consecutive groups of views in turn, each
 *                        group as many views as fit in P pixels (at least
 *                        one), reusing one workspace, so records, pairs and
 *                        contributor bits are sized for one group
 *                        (record_capacity and pair_capacity then count per
 *                        group; the default record capacity is n times the
 *                        group's views).  Results do not depend on it.  When
 *                        the views need more than one group only
 *                        gs_render_candidates and gs_workspace_size (the
 *                        largest group's bytes) accept the view list; the
 *                        other entry points return GS_ERR_ARG. */
typedef struct gs_config {
  int32_t tile_w, tile_h;
  int32_t sem_detach_geometry;
  int32_t px_per_thread;
  int64_t record_capacity;
  int64_t pair_capacity;
  int32_t recompute_bwd;
  int32_t spin_limit;
  int64_t cand_bits_bytes;
  int32_t cand_batch;
  int64_t cand_group_pixels;
} gs_config;

/* Counters read back by gs_read_counters. */
typedef struct gs_counters {
  uint32_t status;      /* bit set of gs_status codes raised on the device (1 << code) */
  uint32_t n_records;   /* visible (view, Gaussian) records (may exceed capacity;
                           the largest group's of a grouped candidate call) */
  uint32_t n_pairs;     /* (tile, Gaussian) pairs (may exceed capacity; idem) */
  uint32_t n_contrib;   /* (pixel, Gaussian) contributions blended by the last forward render */
} gs_counters;

/* Device pointers into a workspace (for inspection and parity tests).  Only
 * host arithmetic: nothing is read from the GPU. */
typedef struct gs_workspace_map {
  void *counters;      /* gs_counters */
  void *rec_uv;        /* float2 [record_capacity]  2D mean (pixels) */
  void *rec_conic;     /* float4 [record_capacity]  (a, b, c, opacity) */
  void *rec_depth;     /* float  [record_capacity]  camera-space z */
  void *rec_rect;      /* short4 [record_capacity]  (x0, x1, y0, y1) inclusive pixels */
  void *rec_gid;       /* int32  [record_capacity]  Gaussian index */
  void *rec_view;      /* int32  [record_capacity]  view index */
  void *pair_tile;     /* uint32 [pair_capacity]    sorted global tile id */
  void *pair_rec;      /* uint32 [pair_capacity]    sorted record index */
  void *tile_ranges;   /* uint2  [total_tiles]      [start, end) into the pair list */
  void *tile_offset;   /* uint32 [n_views + 1]      first global tile id of each view */
  int64_t record_capacity, pair_capacity, total_tiles;
} gs_workspace_map;

/* Workspace bytes for `n_views` cameras (1 for mapping; up to 256 for
 * candidates).  Returns 0 on invalid arguments. */
size_t gs_workspace_size(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg);

/* Fills *map from the workspace base pointer (no device access). */
gs_status gs_workspace_layout(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg,
                              void *ws, gs_workspace_map *map);

/* Projection (Sec. 3.1 "Gaussian Mapping": transform the Gaussians to camera
 * space and project them to the image plane; EWA projection of 3DGS, the
 * prior art the paper adopts).  For every (view, Gaussian) computes the
 * camera-space mean, the 2D mean, the dilated 2D covariance (+0.3 px^2) and
 * its inverse (the conic), the radius ceil(3 sqrt(lambda_max)) and the pixel
 * rectangle of pixels whose centre lies within that radius per axis.  Culls
 * z <= near, non-positive determinant and rectangles outside the image.
 * Visible records are compacted in (view, Gaussian index) order into the
 * workspace.  Resets the workspace status word. */
gs_status gs_project(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg, void *ws,
                     gs_stream_t stream);

/* Binning and front-to-back sort (Sec. 3.1: "sorting them front-to-back";
 * supplement "Sparse Rendering": per tile, batches of the frustum's
 * Gaussians).  Emits one pair per tile of each record's tile rectangle and
 * orders pairs by (view, tile, depth bits, Gaussian index); writes per-tile
 * [start, end) ranges.  Requires a preceding gs_project with the same
 * arguments. */
gs_status gs_bin_sort(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg, void *ws,
                      gs_stream_t stream);

/* Forward render of one view (Eq. 1 with z_i in {c_i, d_i, 1}; Eq. 3 for the
 * sparse top-k semantics; supplement "Sparse Rendering").  Per pixel, the
 * Gaussians whose pixel rectangle holds the pixel are composited front to
 * back with alpha = min(0.99, o exp(-0.5 d^T conic d)), skipped when
 * alpha < 1/255, and the pixel stops before a Gaussian that would take the
 * transmittance below 1e-4.  Outputs (caller-owned device buffers):
 *   rgb [H,W,3], depth [H,W], sil [H,W] (= 1 - final transmittance),
 *   sem [H,W,m] or NULL.
 * Keeps the per-pixel final transmittance and last-contributor index in the
 * workspace for gs_render_bwd.  Requires gs_project + gs_bin_sort with
 * n_views = 1 and the same camera. */
gs_status gs_render_fwd(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws, float *rgb,
                        float *depth, float *sil, float *sem, gs_stream_t stream);

/* Adjoint of gs_render_fwd and gs_project (Sec. 3.1: the rendering is
 * differentiable and optimised end to end; Sec. 6: semantic gradients
 * blocked from geometry).  Upstream gradients with the output shapes of
 * gs_render_fwd (any may be NULL = zero).  Gradients are ACCUMULATED (+=)
 * into g_means [n,3], g_scales [n,3] (w.r.t. linear scales), g_quats [n,4]
 * (w.r.t. the unnormalised quaternion), g_opacity [n], g_rgb [n,3],
 * g_sem_w [n,k].  The transmittance before each contributor is recovered from
 * the stored final transmittance; no per-pixel lists are kept.  Must follow
 * the gs_render_fwd whose outputs it differentiates, with the same workspace. */
gs_status gs_render_bwd(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                        const float *d_rgb, const float *d_depth, const float *d_sil, const float *d_sem,
                        float *g_means, float *g_scales, float *g_quats, float *g_opacity, float *g_rgb,
                        float *g_sem_w, gs_stream_t stream);

/* Forward render of one view fused with the mean-L1 mapping loss (Sec. 3.1:
 * Eq. 1 / Eq. 3 rendering, the L1 colour and depth terms of Eq. 2 without the
 * silhouette mask, plus an L1 term on the semantic distribution):
 *   *loss = mean|rgb - t_rgb| + mean|depth - t_depth| + mean|sem - t_sem|
 * with the targets in the output layouts of gs_render_fwd (t_sem may be NULL
 * to drop the semantic term).  The comparison happens inside the tile kernel:
 * the semantic map need not be written (rgb, depth, sil, sem outputs are
 * optional, NULL to skip).  Per rendered value the workspace keeps two bits
 * (nonzero, negative) of the sign of (rendered - target) for
 * gs_render_bwd_l1, so the per-pixel gradient maps are never materialised.
 * *loss is a device float.  Same preconditions as gs_render_fwd. */
gs_status gs_render_fwd_l1(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                           const float *t_rgb, const float *t_depth, const float *t_sem, float *rgb, float *depth,
                           float *sil, float *sem, float *loss, gs_stream_t stream);

/* Adjoint of gs_render_fwd_l1: accumulates (+=) the gradients of
 * (*loss_scale) * loss into g_* exactly as gs_render_bwd would for upstream
 * gradients sign(x - t) / count.  loss_scale is a DEVICE float (dL/dloss,
 * e.g. the autograd grad_output), read on the stream, so no host
 * synchronisation is needed.  Must follow the gs_render_fwd_l1 it
 * differentiates, with the same workspace. */
gs_status gs_render_bwd_l1(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                           const float *loss_scale, float *g_means, float *g_scales, float *g_quats,
                           float *g_opacity, float *g_rgb, float *g_sem_w, gs_stream_t stream);

/* Batched candidate-view rendering for next-best-view scoring (Sec. 3.2:
 * geometric criterion Eq. 6 from the rendered silhouette, semantic criterion
 * Eq. 7 from the entropy Eq. 4 of the rendered semantic map clipped to
 * [0.001, 1] and renormalised).  Runs projection and binning for all views
 * and one blend launch over every (view, tile); per-pixel maps are never
 * written.  out is a caller-owned device array double[n_views][3]:
 *   out[v][0] = sum_p U(p), U composited by Eq. 1 with z_i = geo_unc[i]
 *               (0 if geo_unc is NULL),
 *   out[v][1] = sum_p H(p) (natural log),
 *   out[v][2] = N_S = number of pixels with S(p) = 0.
 * The softmax normalisations of Eq. 6-8 over candidates are left to the
 * caller.  1 <= n_views <= 256. */
gs_status gs_render_candidates(const gs_scene *scene, const gs_camera *views, int n_views, const gs_config *cfg,
                               void *ws, double *out, gs_stream_t stream);

/* Mean-L1 mapping loss and its gradient (the per-pixel photometric/depth
 * L1 terms of Sec. 3.1 Eq. 2, without the silhouette mask, plus an L1 term on
 * the semantic map): loss = mean|rgb - t_rgb| + mean|depth - t_depth| +
 * mean|sem - t_sem| over npix pixels (sem terms skipped when sem is NULL).
 * Writes d_* = sign(x - t) / count (0 where equal) and *loss (device float).
 * partial is caller scratch of at least 2048 doubles. */
gs_status gs_l1_loss(int64_t npix, int m, const float *rgb, const float *t_rgb, const float *depth,
                     const float *t_depth, const float *sem, const float *t_sem, float *d_rgb, float *d_depth,
                     float *d_sem, float *loss, double *partial, gs_stream_t stream);

/* Number of doubles of the `partial` scratch gs_mapping_loss needs. */
#define GS_MAPPING_LOSS_PARTIALS 2048

/* The mapping objective of Sec. 3.1 on rendered maps (npix pixels, m
 * classes, top-k count k of the map):
 *   sum_p [S(p) > 0.99] (|D(p) - D*(p)| + 0.5 sum_c |C_c(p) - C*_c(p)|)
 *   + mean_p M_H(p) (0.8 D_HD(Q(p) || P(p)) + 0.2 (1 - cos(Q(p), P(p))))
 * with the target distribution Q = t_sem, the rendered P = sem, the entropy
 * mask M_H = [H(Q) < ln k] (Sec. 3.1 "Semantic Loss", Eq. 4), the Hellinger
 * distance D_HD = sqrt(0.5 sum_m (sqrt(Q_m + e) - sqrt(max(P_m, 0) + e))^2),
 * e = 1e-12, and the cosine similarity (0 for a zero norm).  The semantic
 * term is skipped when sem is NULL.  Writes the gradients with respect to
 * rgb [npix][3], depth [npix] and sem [npix][m] (any output may be NULL; the
 * silhouette only masks, so it gets none) and *loss (device float).
 * partial: caller scratch of GS_MAPPING_LOSS_PARTIALS doubles. */
gs_status gs_mapping_loss(int64_t npix, int m, int k, const float *rgb, const float *t_rgb, const float *depth,
                          const float *t_depth, const float *sil, const float *sem, const float *t_sem, float *d_rgb,
                          float *d_depth, float *d_sem, float *loss, double *partial, gs_stream_t stream);

/* Dense-semantic comparator (supplement "Sparse Rendering" and "Runtime
 * Analysis"): gs_render_fwd with every Gaussian carrying a full distribution
 * over all m classes instead of its top-k entries.  sem_dense is a
 * caller-owned device array [n][m] (row-major float; the scene's sparse
 * sem_ids / sem_w are not read for the class map); Eq. 3 blends all m
 * classes of every contributor.  Outputs as gs_render_fwd (sem [H,W,m] or
 * NULL; sem_dense may be NULL only when sem is).  A dense array holding a
 * Gaussian's top-k weights at their ids and zeros elsewhere renders exactly
 * the sparse map.  Same preconditions as gs_render_fwd; the contributor bits
 * must be kept (recompute_bwd = 0), else GS_ERR_UNSUPPORTED. */
gs_status gs_render_fwd_dense(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                              const float *sem_dense, float *rgb, float *depth, float *sil, float *sem,
                              gs_stream_t stream);

/* Forward render of one view fused with the Sec. 3.1 mapping objective of
 * gs_mapping_loss (the silhouette-masked depth / colour L1 sum plus the mean
 * entropy-masked Hellinger + cosine semantic term, Eq. 4, Eq. 5), evaluated
 * inside the tile kernels: the semantic map and its gradient are never
 * written.  Targets in the output layouts of gs_render_fwd; t_sem may be NULL
 * to drop the semantic term.  Outputs rgb, depth, sil are optional (NULL to
 * skip); *loss is a device float.  The workspace keeps, per pixel, the signs
 * of the masked depth / colour errors, and per (Gaussian, entry) the
 * semantic term's gradient with respect to sem_w, for gs_render_bwd_objective.
 * Same preconditions as gs_render_fwd, and in addition:
 *   - cfg->sem_detach_geometry = 1 (the semantic term reaches the semantic
 *     weights only, Sec. 3.1), and the contributor bits are kept
 *     (recompute_bwd = 0);
 *   - the per-pixel class accumulator of a tile fits shared memory in one
 *     chunk (m up to 104 classes at 16x16 tiles with k = 3) and k <= 16.
 * Otherwise returns GS_ERR_UNSUPPORTED before any GPU work: render with
 * gs_render_fwd and evaluate gs_mapping_loss on the maps instead. */
gs_status gs_render_fwd_objective(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                                  const float *t_rgb, const float *t_depth, const float *t_sem, float *rgb,
                                  float *depth, float *sil, float *loss, gs_stream_t stream);

/* Adjoint of gs_render_fwd_objective: accumulates (+=) the gradients of
 * (*loss_scale) * loss into g_* (layouts of gs_render_bwd), equal to
 * gs_render_bwd with the upstream gradients gs_mapping_loss writes.
 * loss_scale is a DEVICE float read on the stream.  Must follow the
 * gs_render_fwd_objective it differentiates, with the same workspace and
 * configuration. */
gs_status gs_render_bwd_objective(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                                  const float *loss_scale, float *g_means, float *g_scales, float *g_quats,
                                  float *g_opacity, float *g_rgb, float *g_sem_w, gs_stream_t stream);

/* Scoring tail of the candidate renders (Sec. 3.2, Eq. 6-8), on the device
 * and stream-ordered (graph-capturable after gs_render_candidates).  Over the
 * n_views candidates given:
 *   I_geo = softmax(log N_S) = N_S / sum N_S (all 0 when no view has N_S > 0)
 *   I_sem = softmax(sum_p H)
 *   I     = (1 - softmax(l)) I_geo I_sem,  l = |position - current|
 * softmaxes in double with the maximum subtracted.  Device inputs: sums
 * [n_views][3] as written by gs_render_candidates (sum U, sum H, N_S), npix
 * [n_views] pixels per view, positions [n_views][3] candidate positions,
 * current [3] the camera's position.  Device outputs: scores [n_views][4] =
 * (I, I_geo, I_sem, 1 - softmax(l)); keep [n_views] = 1 unless
 * N_S < prune_frac * npix (the pool's pruning rule, prune_frac = 0.005 in
 * the paper); *best = index of the largest I among kept views (lowest index
 * on ties), -1 when none is kept.  0 <= prune_frac <= 1. */
gs_status gs_score_candidates(int n_views, const double *sums, const int32_t *npix, const float *positions,
                              const float *current, double prune_frac, double *scores, int32_t *keep,
                              int32_t *best, gs_stream_t stream);

/* Host: candidate cameras at n_positions positions (host [n_positions][3])
 * times n_dirs viewing directions, the points of an n_dirs-point Fibonacci
 * lattice on the unit sphere (Sec. 3.2 "Exploration Strategy": v2 = 5 in the
 * coarse stage, 15 in the fine one): direction i has height
 * z = 1 - (2 i + 1) / n_dirs and azimuth i times the golden angle
 * pi (3 - sqrt 5).  Camera rows are right = d x (0, 0, 1) normalised,
 * down = d x right, forward = d (OpenCV axes, world z up); principal point
 * at the image centre.  Writes out[p * n_dirs + i] (host array). */
gs_status gs_candidate_poses(int n_positions, const float *positions, int n_dirs, int width, int height, float fx,
                             float fy, float near_plane, gs_camera *out);

/* Host: candidate positions on a lattice of spacing `step` (v1: 1 m coarse,
 * 0.5 m fine) over newly freed space.  For every voxel centre (host
 * [n_voxels][3]) within `band` of one of the n_heights heights h, the
 * lattice point (round(x / step) step, round(y / step) step, h) is a
 * candidate; duplicates are merged and the points written in ascending
 * (i, j, height index) order to out (host [capacity][3]).  Returns the number
 * of distinct points (writing at most capacity of them), or -1 on invalid
 * arguments. */
int64_t gs_candidate_positions(int64_t n_voxels, const float *centres, float step, int n_heights,
                               const float *heights, float band, float *out, int64_t capacity);

/* Sparse semantic representation, initialisation (Sec. 3.1 "Sparse Semantic
 * Representation"): for each of n new Gaussians, the k classes of highest
 * probability in its observed distribution, row rows[i] of probs
 * ([*][m] device array; rows NULL: row i), written as ids [n][k] (int32,
 * descending probability, the lower class id first on ties, NaN ranked
 * below every number) and w [n][k] (the probabilities as observed, not
 * renormalised).  1 <= k <= min(m, 16).  Row indices are the caller's to
 * keep in range. */
gs_status gs_topk_init(int64_t n, int m, int k, const float *probs, const int64_t *rows, int32_t *ids, float *w,
                       gs_stream_t stream);

/* Update of the sparse representation from a new observation with the ids
 * fixed: w[i][l] = probs[rows[i]][ids[i][l]] (entries whose id is outside
 * [0, m) are left unchanged). */
gs_status gs_topk_gather(int64_t n, int m, int k, const float *probs, const int64_t *rows, const int32_t *ids,
                         float *w, gs_stream_t stream);

/* Exploration Map (Sec. 3.2, 5 cm voxels in the paper): a voxel grid with
 * origin (world metres, the corner of voxel (0, 0, 0)), voxel edge length
 * and size; voxel (x, y, z) has linear index (z ny + y) nx + x. */
typedef struct {
  float origin[3];
  float voxel;
  int32_t nx, ny, nz;
} gs_voxel_grid;

/* uint32 words of a grid's state array (2 bits per voxel, 16 per word: bit
 * 2j seen free, bit 2j + 1 seen occupied); -1 for an invalid grid.  A new
 * map is all zero (unknown). */
int64_t gs_voxel_words(const gs_voxel_grid *grid);

/* uint32 words of the scratch gs_voxel_new_free needs; -1 if invalid. */
int64_t gs_voxel_scratch_words(const gs_voxel_grid *grid);

/* Updates the state (device, gs_voxel_words words) from one depth frame
 * (device [height][width] float, camera-space z as rendered by
 * gs_render_fwd) seen by cam: for every stride-th column and row, the
 * segment from the camera centre to the back-projected point marks every
 * voxel it passes free and the voxel holding the point occupied (only bits
 * are set: the result does not depend on the order of the rays).  Depths
 * above max_depth are cut at max_depth and mark nothing occupied; depths
 * that are not positive and finite are skipped.  Parts of a segment outside
 * the grid are ignored. */
gs_status gs_voxel_update(const gs_voxel_grid *grid, uint32_t *state, const float *depth, const gs_camera *cam,
                          int stride, float max_depth, gs_stream_t stream);

/* The voxels newly freed between two states (free and not occupied in cur,
 * unknown in prev): their centres written in ascending voxel index to
 * centres (device [capacity][3]), their number (which may exceed capacity)
 * to *count (device uint32).  scratch: device, gs_voxel_scratch_words
 * words. */
gs_status gs_voxel_new_free(const gs_voxel_grid *grid, const uint32_t *prev, const uint32_t *cur, uint32_t *scratch,
                            float *centres, int64_t capacity, uint32_t *count, gs_stream_t stream);

/* Work counters of the blend passes over the views binned in `ws` (call
 * after gs_project and gs_bin_sort with the same arguments), for roofline
 * figures; not meant for the timed path.  Per pixel of every view:
 *   n_eval      (pixel, Gaussian) pairs whose pixel rectangle holds the
 *               pixel, up to and including the pair that stops the pixel's
 *               compositing (T (1 - alpha) < 1e-4): the evaluations of the
 *               per-pixel definition of Eq. 1;
 *   n_eval_box  of those, the pairs inside the Gaussian's alpha box (the
 *               pairs the blend kernels evaluate; outside, alpha < 1/255);
 *   n_contrib   pairs blended (alpha >= 1/255, before the stop);
 *   n_touched   (pixel, class) entries of the Eq. 3 distribution above the
 *               0.001 clip floor of Eq. 7 (the logarithms of the entropy);
 *   n_pixels    pixels inside the views.
 * `out` is a DEVICE pointer (8-byte aligned), overwritten.  per_pixel
 * (optional DEVICE uint32 [height][width][2], single view only, else
 * GS_ERR_ARG) receives each pixel's (n_eval, n_contrib). */
typedef struct gs_work_counts {
  uint64_t n_eval, n_eval_box, n_contrib, n_touched, n_pixels;
} gs_work_counts;
gs_status gs_count_work(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg, void *ws,
                        gs_work_counts *out, uint32_t *per_pixel, gs_stream_t stream);

/* Bytes of the fixed device scratch array used by gs_render_fwd_noalloc. */
#define GS_NOALLOC_SCRATCH_BYTES (32u << 20)

/* No-allocation variant of one forward render (the paper has no counterpart:
 * this is an interface for callers of this library).
 *
 * Some callers cannot allocate device memory: plug-in hosts that own all
 * device memory and give their plug-ins none, and real-time loops that must
 * never block inside an allocator (cudaMalloc and cudaFree may synchronise
 * the device).  This entry point
 * runs the same kernels as gs_project + gs_bin_sort + gs_render_fwd for one
 * view, but its workspace is a fixed device array of
 * GS_NOALLOC_SCRATCH_BYTES inside the library, so it calls no cudaMalloc,
 * cudaFree or other allocating routine.  Every GPU that loads the library
 * holds that array until the process exits.
 *   - Arguments are those of gs_render_fwd without the workspace; outputs
 *     (rgb, depth, sil, sem; any may be NULL) are caller-owned device buffers.
 *   - Returns GS_ERR_TOO_LARGE, before any GPU work, when the workspace these
 *     sizes and capacities need (gs_workspace_size with n_views = 1) exceeds
 *     GS_NOALLOC_SCRATCH_BYTES.
 *   - The first call on each device looks up the array's device address
 *     (with that device current) and caches it; make that first call before
 *     any stream capture.  The cached address belongs to the device's primary
 *     context: after cudaDeviceReset of that device, do not call this entry
 *     point again in the same process.
 *   - All calls share the one array, which keeps the previous call's
 *     contents; the chain clears what must start at zero (counters, status).
 *     Calls that overlap on the GPU (other streams, other host threads) race
 *     on the array and must be serialised by the caller.
 *   - counters_out (optional DEVICE pointer) receives the chain's counters,
 *     including the capacity status bit, at the end of the chain. */
gs_status gs_render_fwd_noalloc(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, float *rgb,
                                float *depth, float *sil, float *sem, gs_counters *counters_out,
                                gs_stream_t stream);

/* Testing hooks (host only; no device work).  Grid sizes of the grid-stride
 * kernels follow the multiprocessor count of the current device, which the
 * library queries once per device (cudaDevAttrMultiProcessorCount) and
 * caches; one process may drive several devices.
 *   gs_testing_set_sm_query  replaces that query by `query` (NULL restores
 *                            the device query), so host tests can check the
 *                            grids for any SM count without a GPU;
 *   gs_testing_grid          the grid (CTAs) the library would launch for
 *                            one of the kernels below on the current device
 *                            (0 when the SM count is unknown, -1 for an
 *                            unknown id). */
enum {
  GS_GRID_EMIT_CHUNKS = 0, /* chunks of the pair-emission count pass: 2 per SM, at most 1024 */
  GS_GRID_EMIT_WRITE = 1,  /* pair-emission write pass: 8 per SM */
  GS_GRID_SORT_RESET = 2,  /* radix-sort reset and digit histogram: 2 per SM */
  GS_GRID_RANGES = 3,      /* tile-range marking: 4 per SM */
  GS_GRID_ZERO_GRAD = 4    /* 2D-gradient clear of the adjoint: 2 per SM */
};
void gs_testing_set_sm_query(int (*query)(void));
int64_t gs_testing_grid(int which);

/* Synchronises `stream`, then copies the workspace counters to *out (host).
 * Returns the first device error recorded (GS_ERR_CAPACITY, GS_ERR_TIMEOUT)
 * or GS_OK. */
gs_status gs_read_counters(void *ws, gs_counters *out, gs_stream_t stream);

/* Static description of a status code. */
const char *gs_status_string(gs_status s);

#ifdef __cplusplus
}
#endif
#endif /* GS_H_ */
