/*
 * gs_oracle.c -- plain, slow CPU oracle for the semantic Gaussian rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * What it computes (ActiveSGM, arXiv 2506.00225):
 *   - per-Gaussian projection of an anisotropic 3D Gaussian to a 2D conic
 *     (Sec. 3.1 "Gaussian Mapping": transform to camera space, project to the
 *     image plane; the EWA formula itself is the 3DGS prior art the paper
 *     builds on), its pixel rectangle and tile rectangle;
 *   - per pixel, brute-force depth-ordered compositing of Eq. 1 for colour,
 *     depth, silhouette (z_i in {c_i, d_i, 1}) and of Eq. 3 for the sparse
 *     top-k semantic distribution, with an optional scalar channel (geometric
 *     uncertainty) composited the same way;
 *   - the hand-derived adjoint of both (gradients w.r.t. means, scales,
 *     quaternions, opacities, colours and sparse semantic weights), with the
 *     semantic-to-geometry gradient block of Sec. 3.1 "Semantic Loss";
 *   - candidate-view reductions: N_S of Eq. 6 (pixels with S = 0), the sum of
 *     per-pixel entropies (Eq. 4) of the clipped-to-[0.001, 1], renormalised
 *     semantic map of Eq. 7, and the summed composited uncertainty.
 *
 * The same source builds twice: REAL = float (decisions taken in the
 * kernel's precision, no FMA contraction: compile with -ffp-contract=off)
 * and REAL = double (for finite-difference checks of the adjoint).
 *
 * Camera array layout (REAL cam[17]): fx, fy, cx, cy, near, w2c[12] with
 * w2c row-major [R | t] (OpenCV axes: x right, y down, z forward).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORC_DOUBLE
typedef double real;
#define R_EXP exp
#define R_SQRT sqrt
#define R_CEIL ceil
#define R_FLOOR floor
#define R_LOG log
#define R_ISFINITE isfinite
#define SFX(name) name##_f64
#else
typedef float real;
#define R_EXP expf
#define R_SQRT sqrtf
#define R_CEIL ceilf
#define R_FLOOR floorf
#define R_LOG logf
#define R_ISFINITE isfinite
#define SFX(name) name##_f32
#endif

/* Constants of the per-pixel opacity rule (3DGS prior art the paper adopts
 * via SplaTAM): opacity cap, skip threshold, transmittance stop, 2D dilation,
 * radius multiplier, eigenvalue floor, frustum clamp factor. */
#define ALPHA_MAX ((real)0.99)
#define ALPHA_MIN ((real)1 / (real)255)
#define T_STOP ((real)0.0001)
#define DILATION ((real)0.3)
#define SIGMA_MUL ((real)3)
#define EIG_FLOOR ((real)0.1)
#define FRUSTUM_CLAMP ((real)1.3)
/* relative margin under which a threshold decision counts as "near" */
#define MARGIN_REL 1e-5

/* ------------------------------------------------------------------------ */
/* Projection                                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  int visible;
  real tx, ty, tz;          /* camera-space mean */
  real rxc, ryc;            /* clamped tx/tz, ty/tz */
  int clampx, clampy;       /* 1 if the clamp was active */
  real qn, w, x, y, z;      /* |q| and the unit quaternion */
  real Rq[9];               /* rotation of the unit quaternion */
  real Mq[9];               /* Rq * diag(s) */
  real S3[9];               /* 3D covariance (full symmetric) */
  real J00, J02, J11, J12;
  real T[6];                /* J W, 2x3 */
  real A, B, C;             /* dilated 2D covariance */
  real det, inv;
  real ca, cb, cc;          /* conic */
  real radius;
  real u, v;                /* 2D mean (pixels) */
  int x0, x1, y0, y1;       /* inclusive pixel rectangle (clamped) */
  int tx0, tx1, ty0, ty1;   /* inclusive tile rectangle */
  int ntiles;
} proj_t;

static void project_one(const real *m, const real *s, const real *q, const real *cam,
                        int W, int H, int tw, int th, proj_t *p) {
  memset(p, 0, sizeof(*p));
  const real fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3], znear = cam[4];
  const real *V = cam + 5; /* w2c */
  /* camera-space mean t = R m + t_c, summed left to right */
  p->tx = ((V[0] * m[0] + V[1] * m[1]) + V[2] * m[2]) + V[3];
  p->ty = ((V[4] * m[0] + V[5] * m[1]) + V[6] * m[2]) + V[7];
  p->tz = ((V[8] * m[0] + V[9] * m[1]) + V[10] * m[2]) + V[11];
  if (!(R_ISFINITE(p->tx) && R_ISFINITE(p->ty) && R_ISFINITE(p->tz))) return;
  if (!(p->tz > znear)) return;
  /* unit quaternion */
  real n2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
  if (!(n2 > 0) || !R_ISFINITE(n2)) return;
  p->qn = R_SQRT(n2);
  p->w = q[0] / p->qn; p->x = q[1] / p->qn; p->y = q[2] / p->qn; p->z = q[3] / p->qn;
  real w = p->w, x = p->x, y = p->y, z = p->z;
  real xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  real wx = w * x, wy = w * y, wz = w * z;
  real *R = p->Rq;
  R[0] = (real)1 - (real)2 * (yy + zz); R[1] = (real)2 * (xy - wz); R[2] = (real)2 * (xz + wy);
  R[3] = (real)2 * (xy + wz); R[4] = (real)1 - (real)2 * (xx + zz); R[5] = (real)2 * (yz - wx);
  R[6] = (real)2 * (xz - wy); R[7] = (real)2 * (yz + wx); R[8] = (real)1 - (real)2 * (xx + yy);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) p->Mq[i * 3 + j] = R[i * 3 + j] * s[j];
  /* Sigma3 = M M^T */
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      const real *a = p->Mq + i * 3, *b = p->Mq + j * 3;
      real v = (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
      p->S3[i * 3 + j] = v;
      p->S3[j * 3 + i] = v;
    }
  /* Jacobian of the pinhole projection at the (frustum-clamped) mean */
  real limx = FRUSTUM_CLAMP * (((real)0.5 * (real)W) / fx);
  real limy = FRUSTUM_CLAMP * (((real)0.5 * (real)H) / fy);
  real rx = p->tx / p->tz, ry = p->ty / p->tz;
  p->rxc = rx < -limx ? -limx : (rx > limx ? limx : rx);
  p->ryc = ry < -limy ? -limy : (ry > limy ? limy : ry);
  p->clampx = (rx < -limx) || (rx > limx);
  p->clampy = (ry < -limy) || (ry > limy);
  real txc = p->rxc * p->tz, tyc = p->ryc * p->tz;
  real tz2 = p->tz * p->tz;
  p->J00 = fx / p->tz;
  p->J02 = -(fx * txc) / tz2;
  p->J11 = fy / p->tz;
  p->J12 = -(fy * tyc) / tz2;
  /* T = J W (W = camera rotation) */
  for (int j = 0; j < 3; ++j) {
    p->T[j] = p->J00 * V[0 + j] + p->J02 * V[8 + j];
    p->T[3 + j] = p->J11 * V[4 + j] + p->J12 * V[8 + j];
  }
  /* U = T Sigma3, Sigma2 = U T^T */
  real U[6];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 3; ++j)
      U[a * 3 + j] = (p->T[a * 3 + 0] * p->S3[0 * 3 + j] + p->T[a * 3 + 1] * p->S3[1 * 3 + j]) +
                     p->T[a * 3 + 2] * p->S3[2 * 3 + j];
  p->A = ((U[0] * p->T[0] + U[1] * p->T[1]) + U[2] * p->T[2]) + DILATION;
  p->B = (U[0] * p->T[3] + U[1] * p->T[4]) + U[2] * p->T[5];
  p->C = ((U[3] * p->T[3] + U[4] * p->T[4]) + U[5] * p->T[5]) + DILATION;
  if (!(R_ISFINITE(p->A) && R_ISFINITE(p->B) && R_ISFINITE(p->C))) return;
  p->det = p->A * p->C - p->B * p->B;
  if (!(p->det > 0)) return;
  p->inv = (real)1 / p->det;
  p->ca = p->C * p->inv;
  p->cb = -p->B * p->inv;
  p->cc = p->A * p->inv;
  real mid = (real)0.5 * (p->A + p->C);
  real disc = mid * mid - p->det;
  real lam = mid + R_SQRT(disc > EIG_FLOOR ? disc : EIG_FLOOR);
  p->radius = R_CEIL(SIGMA_MUL * R_SQRT(lam));
  p->u = (fx * p->tx) / p->tz + cx;
  p->v = (fy * p->ty) / p->tz + cy;
  if (!(R_ISFINITE(p->u) && R_ISFINITE(p->v))) return;
  /* pixel x is covered iff its centre x+0.5 lies within radius of u */
  real xlo = R_CEIL((p->u - (real)0.5) - p->radius);
  real xhi = R_FLOOR((p->u - (real)0.5) + p->radius);
  real ylo = R_CEIL((p->v - (real)0.5) - p->radius);
  real yhi = R_FLOOR((p->v - (real)0.5) + p->radius);
  if (xlo < 0) xlo = 0;
  if (ylo < 0) ylo = 0;
  if (xhi > (real)(W - 1)) xhi = (real)(W - 1);
  if (yhi > (real)(H - 1)) yhi = (real)(H - 1);
  if (!(xlo <= xhi) || !(ylo <= yhi)) return;
  p->x0 = (int)xlo; p->x1 = (int)xhi; p->y0 = (int)ylo; p->y1 = (int)yhi;
  p->tx0 = p->x0 / tw; p->tx1 = p->x1 / tw; p->ty0 = p->y0 / th; p->ty1 = p->y1 / th;
  p->ntiles = (p->tx1 - p->tx0 + 1) * (p->ty1 - p->ty0 + 1);
  p->visible = 1;
}

/* Project all n Gaussians.  Outputs (any may be NULL):
 * uv[n,2], conic[n,3], depth[n], radius[n], rect[n,4] (x0,x1,y0,y1),
 * trect[n,4] (tx0,tx1,ty0,ty1), ntiles[n], visible[n]. */
void SFX(orc_project)(int n, const real *means, const real *scales, const real *quats,
                      const real *cam, int W, int H, int tw, int th,
                      real *uv, real *conic, real *depth, real *radius,
                      int *rect, int *trect, int *ntiles, int *visible) {
  for (int i = 0; i < n; ++i) {
    proj_t p;
    project_one(means + 3 * i, scales + 3 * i, quats + 4 * i, cam, W, H, tw, th, &p);
    if (uv) { uv[2 * i] = p.u; uv[2 * i + 1] = p.v; }
    if (conic) { conic[3 * i] = p.ca; conic[3 * i + 1] = p.cb; conic[3 * i + 2] = p.cc; }
    if (depth) depth[i] = p.tz;
    if (radius) radius[i] = p.radius;
    if (rect) { rect[4 * i] = p.x0; rect[4 * i + 1] = p.x1; rect[4 * i + 2] = p.y0; rect[4 * i + 3] = p.y1; }
    if (trect) { trect[4 * i] = p.tx0; trect[4 * i + 1] = p.tx1; trect[4 * i + 2] = p.ty0; trect[4 * i + 3] = p.ty1; }
    if (ntiles) ntiles[i] = p.visible ? p.ntiles : 0;
    if (visible) visible[i] = p.visible;
  }
}

/* ------------------------------------------------------------------------ */
/* Per-pixel compositing                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n, k, m;
  const real *means, *scales, *quats, *opacity, *rgb, *sem_w, *unc;
  const int *sem_ids;
} scene_t;

typedef struct { int gid; real depth; } dkey_t;

static int cmp_depth(const void *a, const void *b) {
  const dkey_t *x = (const dkey_t *)a, *y = (const dkey_t *)b;
  if (x->depth < y->depth) return -1;
  if (x->depth > y->depth) return 1;
  return (x->gid > y->gid) - (x->gid < y->gid);
}

/* Visible Gaussians sorted by (depth, gid): every pixel's candidate list is
 * this order restricted to the Gaussians whose rectangle holds the pixel. */
typedef struct {
  int nv;
  int *order;     /* gids, depth order */
  proj_t *proj;   /* indexed by gid */
  int *row_start; /* CSR over rows: Gaussians (depth order) covering row y */
  int *row_items;
} view_t;

static void view_build(const scene_t *sc, const real *cam, int W, int H, view_t *vw) {
  vw->proj = (proj_t *)malloc(sizeof(proj_t) * (size_t)(sc->n > 0 ? sc->n : 1));
  dkey_t *keys = (dkey_t *)malloc(sizeof(dkey_t) * (size_t)(sc->n > 0 ? sc->n : 1));
  int nv = 0;
  for (int i = 0; i < sc->n; ++i) {
    project_one(sc->means + 3 * i, sc->scales + 3 * i, sc->quats + 4 * i, cam, W, H, 16, 16, &vw->proj[i]);
    if (vw->proj[i].visible) { keys[nv].gid = i; keys[nv].depth = vw->proj[i].tz; ++nv; }
  }
  qsort(keys, (size_t)nv, sizeof(dkey_t), cmp_depth);
  vw->nv = nv;
  vw->order = (int *)malloc(sizeof(int) * (size_t)(nv > 0 ? nv : 1));
  for (int i = 0; i < nv; ++i) vw->order[i] = keys[i].gid;
  free(keys);
  vw->row_start = (int *)calloc((size_t)H + 1, sizeof(int));
  for (int i = 0; i < nv; ++i) {
    const proj_t *p = &vw->proj[vw->order[i]];
    for (int y = p->y0; y <= p->y1; ++y) vw->row_start[y + 1]++;
  }
  for (int y = 0; y < H; ++y) vw->row_start[y + 1] += vw->row_start[y];
  int total = vw->row_start[H];
  vw->row_items = (int *)malloc(sizeof(int) * (size_t)(total > 0 ? total : 1));
  int *fill = (int *)malloc(sizeof(int) * (size_t)H);
  for (int y = 0; y < H; ++y) fill[y] = vw->row_start[y];
  for (int i = 0; i < nv; ++i) {
    int g = vw->order[i];
    const proj_t *p = &vw->proj[g];
    for (int y = p->y0; y <= p->y1; ++y) vw->row_items[fill[y]++] = g;
  }
  free(fill);
}

static void view_free(view_t *vw) {
  free(vw->proj); free(vw->order); free(vw->row_start); free(vw->row_items);
}

/* One contributor of a pixel, kept for the adjoint. */
typedef struct { int gid; real alpha, a, G, T, dx, dy; } contrib_t;

typedef struct {
  real rgb[3], depth, unc, T;
  int n_contrib;
  long n_eval;
  int flag;        /* 1 if a threshold decision was within the relative margin */
} pix_t;

/* Composite pixel (x, y).  sem (length m) is accumulated if non-NULL;
 * contributors are recorded if list != NULL (capacity cap). */
static void composite_pixel(const scene_t *sc, const view_t *vw, int x, int y, real *sem,
                            pix_t *out, contrib_t *list, int cap) {
  real T = 1, cr = 0, cg = 0, cb = 0, d = 0, u = 0;
  int nc = 0, flag = 0;
  long ne = 0;
  const real px = (real)x + (real)0.5, py = (real)y + (real)0.5;
  for (int it = vw->row_start[y]; it < vw->row_start[y + 1]; ++it) {
    int g = vw->row_items[it];
    const proj_t *p = &vw->proj[g];
    if (x < p->x0 || x > p->x1) continue;
    ++ne;
    real dx = p->u - px, dy = p->v - py;
    real power = -(real)0.5 * (p->ca * (dx * dx) + p->cc * (dy * dy)) - p->cb * (dx * dy);
    if (power > 0) continue;
    real G = R_EXP(power);
    real a = sc->opacity[g] * G;
    real alpha = a < ALPHA_MAX ? a : ALPHA_MAX;
    if (fabs((double)a - (double)ALPHA_MIN) <= MARGIN_REL * (double)ALPHA_MIN) flag |= 1;
    if (fabs((double)a - (double)ALPHA_MAX) <= MARGIN_REL) flag |= 2;
    if (alpha < ALPHA_MIN) continue;
    real Tn = T * ((real)1 - alpha);
    if (fabs((double)Tn - (double)T_STOP) <= MARGIN_REL * (double)T_STOP) flag |= 1;
    if (Tn < T_STOP) break;
    real w = alpha * T;
    cr += w * sc->rgb[3 * g]; cg += w * sc->rgb[3 * g + 1]; cb += w * sc->rgb[3 * g + 2];
    d += w * p->tz;
    if (sc->unc) u += w * sc->unc[g];
    if (sem)
      for (int j = 0; j < sc->k; ++j) sem[sc->sem_ids[g * sc->k + j]] += w * sc->sem_w[g * sc->k + j];
    if (list && nc < cap) {
      contrib_t *c = &list[nc];
      c->gid = g; c->alpha = alpha; c->a = a; c->G = G; c->T = T; c->dx = dx; c->dy = dy;
    }
    ++nc;
    T = Tn;
  }
  out->rgb[0] = cr; out->rgb[1] = cg; out->rgb[2] = cb;
  out->depth = d; out->unc = u; out->T = T; out->n_contrib = nc; out->n_eval = ne; out->flag = flag;
}

#define SCENE_FROM_ARGS                                                           \
  scene_t sc = {n, k, m, means, scales, quats, opacity, rgb, sem_w, unc, sem_ids};

/* Forward render of rows y_begin, y_begin + y_step, ... < y_end (the full
 * image for 0, H, 1).  Outputs: rgb[H,W,3], depth[H,W], sil[H,W]
 * (= 1 - T_final), unc_img[H,W] (if unc given and unc_img non-NULL),
 * sem[H,W,m] (if non-NULL), T_final[H,W], n_contrib[H,W], n_eval[H,W],
 * flag[H,W].  stats[2] = {N_eval, N_contrib} summed over pixels. */
void SFX(orc_render)(int n, int k, int m, const real *means, const real *scales, const real *quats,
                     const real *opacity, const real *rgb, const int *sem_ids, const real *sem_w,
                     const real *unc, const real *cam, int W, int H,
                     real *out_rgb, real *out_depth, real *out_sil, real *out_unc, real *out_sem,
                     real *out_T, int *out_nc, int *out_ne, int *out_flag, long *stats, int y_begin, int y_end,
                     int y_step) {
  SCENE_FROM_ARGS
  view_t vw;
  view_build(&sc, cam, W, H, &vw);
  long ne = 0, ncs = 0;
  if (y_step < 1) y_step = 1;
  if (y_end > H || y_end < 0) y_end = H;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : ne, ncs)
  for (int y = y_begin; y < y_end; y += y_step) {
    for (int x = 0; x < W; ++x) {
      size_t pid = (size_t)y * W + x;
      real *sem = out_sem ? out_sem + pid * m : NULL;
      if (sem) memset(sem, 0, sizeof(real) * (size_t)m);
      pix_t o;
      composite_pixel(&sc, &vw, x, y, sem, &o, NULL, 0);
      if (out_rgb) { out_rgb[3 * pid] = o.rgb[0]; out_rgb[3 * pid + 1] = o.rgb[1]; out_rgb[3 * pid + 2] = o.rgb[2]; }
      if (out_depth) out_depth[pid] = o.depth;
      if (out_sil) out_sil[pid] = (real)1 - o.T;
      if (out_unc) out_unc[pid] = o.unc;
      if (out_T) out_T[pid] = o.T;
      if (out_nc) out_nc[pid] = o.n_contrib;
      if (out_ne) out_ne[pid] = (int)o.n_eval;
      if (out_flag) out_flag[pid] = o.flag;
      ne += o.n_eval;
      ncs += o.n_contrib;
    }
  }
  if (stats) { stats[0] = ne; stats[1] = ncs; }
  view_free(&vw);
}

/* Forward render of a list of pixels (px[i], py[i]); outputs are indexed by
 * list position with the same per-pixel layouts as orc_render.  Candidate
 * lists come from testing every visible Gaussian's rectangle. */
void SFX(orc_render_pixels)(int n, int k, int m, const real *means, const real *scales, const real *quats,
                            const real *opacity, const real *rgb, const int *sem_ids, const real *sem_w,
                            const real *unc, const real *cam, int W, int H, int npix, const int *pxs,
                            const int *pys, real *out_rgb, real *out_depth, real *out_sil, real *out_unc,
                            real *out_sem, real *out_T, int *out_nc, int *out_flag) {
  SCENE_FROM_ARGS
  view_t vw;
  view_build(&sc, cam, W, H, &vw);
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < npix; ++i) {
    real *sem = out_sem ? out_sem + (size_t)i * m : NULL;
    if (sem) memset(sem, 0, sizeof(real) * (size_t)m);
    pix_t o;
    composite_pixel(&sc, &vw, pxs[i], pys[i], sem, &o, NULL, 0);
    if (out_rgb) { out_rgb[3 * i] = o.rgb[0]; out_rgb[3 * i + 1] = o.rgb[1]; out_rgb[3 * i + 2] = o.rgb[2]; }
    if (out_depth) out_depth[i] = o.depth;
    if (out_sil) out_sil[i] = (real)1 - o.T;
    if (out_unc) out_unc[i] = o.unc;
    if (out_T) out_T[i] = o.T;
    if (out_nc) out_nc[i] = o.n_contrib;
    if (out_flag) out_flag[i] = o.flag;
  }
  view_free(&vw);
}

/* ------------------------------------------------------------------------ */
/* Adjoint                                                                   */
/* ------------------------------------------------------------------------ */

/* Chain the 2D gradients of one Gaussian (du, dv, dconic, ddepth) through
 * the projection to means, linear scales and quaternions. */
static void project_adjoint(const proj_t *p, const real *s, const real *cam, real du, real dv,
                            real dca, real dcb, real dcc, real dz, real *gm, real *gs, real *gq) {
  const real fx = cam[0], fy = cam[1];
  const real *V = cam + 5;
  /* conic = inverse of [[A,B],[B,C]]: ca = C/det, cb = -B/det, cc = A/det */
  real inv = p->inv, inv2 = inv * inv;
  real dinv = dca * p->C - dcb * p->B + dcc * p->A;
  real dA = dcc * inv - dinv * p->C * inv2;
  real dB = -dcb * inv + dinv * (real)2 * p->B * inv2;
  real dC = dca * inv - dinv * p->A * inv2;
  /* A = T0 S T0^T, B = T0 S T1^T, C = T1 S T1^T */
  const real *T = p->T, *S = p->S3;
  real ST0[3], ST1[3];
  for (int i = 0; i < 3; ++i) {
    ST0[i] = S[i * 3 + 0] * T[0] + S[i * 3 + 1] * T[1] + S[i * 3 + 2] * T[2];
    ST1[i] = S[i * 3 + 0] * T[3] + S[i * 3 + 1] * T[4] + S[i * 3 + 2] * T[5];
  }
  real dT[6];
  for (int i = 0; i < 3; ++i) {
    dT[i] = (real)2 * dA * ST0[i] + dB * ST1[i];
    dT[3 + i] = (real)2 * dC * ST1[i] + dB * ST0[i];
  }
  /* dL/dSigma3 (as a full matrix), then symmetrised for Sigma3 = M M^T */
  real G[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      G[i * 3 + j] = dA * T[i] * T[j] + dB * T[i] * T[3 + j] + dC * T[3 + i] * T[3 + j];
  real dM[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      real acc = 0;
      for (int l = 0; l < 3; ++l) acc += (G[i * 3 + l] + G[l * 3 + i]) * p->Mq[l * 3 + j];
      dM[i * 3 + j] = acc;
    }
  real dR[9];
  for (int j = 0; j < 3; ++j) {
    real acc = 0;
    for (int i = 0; i < 3; ++i) {
      acc += dM[i * 3 + j] * p->Rq[i * 3 + j];
      dR[i * 3 + j] = dM[i * 3 + j] * s[j];
    }
    gs[j] += acc;
  }
  /* rotation of the unit quaternion (w,x,y,z) */
  real w = p->w, x = p->x, y = p->y, z = p->z;
  real dw = (real)2 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  real dxq = (real)2 * (y * dR[1] + z * dR[2] + y * dR[3] - (real)2 * x * dR[4] - w * dR[5] + z * dR[6] +
                        w * dR[7] - (real)2 * x * dR[8]);
  real dyq = (real)2 * (-(real)2 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                        z * dR[7] - (real)2 * y * dR[8]);
  real dzq = (real)2 * (-(real)2 * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - (real)2 * z * dR[4] +
                        y * dR[5] + x * dR[6] + y * dR[7]);
  real dot = w * dw + x * dxq + y * dyq + z * dzq;
  gq[0] += (dw - w * dot) / p->qn;
  gq[1] += (dxq - x * dot) / p->qn;
  gq[2] += (dyq - y * dot) / p->qn;
  gq[3] += (dzq - z * dot) / p->qn;
  /* T = J W */
  real dJ00 = dT[0] * V[0] + dT[1] * V[1] + dT[2] * V[2];
  real dJ02 = dT[0] * V[8] + dT[1] * V[9] + dT[2] * V[10];
  real dJ11 = dT[3] * V[4] + dT[4] * V[5] + dT[5] * V[6];
  real dJ12 = dT[3] * V[8] + dT[4] * V[9] + dT[5] * V[10];
  real tz = p->tz, tz2 = tz * tz, tz3 = tz2 * tz;
  real dtx = 0, dty = 0, dtz = dz;
  dtz += dJ00 * (-fx / tz2) + dJ11 * (-fy / tz2);
  if (!p->clampx) { dtx += dJ02 * (-fx / tz2); dtz += dJ02 * ((real)2 * fx * p->tx / tz3); }
  else { dtz += dJ02 * (fx * p->rxc / tz2); }
  if (!p->clampy) { dty += dJ12 * (-fy / tz2); dtz += dJ12 * ((real)2 * fy * p->ty / tz3); }
  else { dtz += dJ12 * (fy * p->ryc / tz2); }
  /* u = fx tx / tz + cx, v = fy ty / tz + cy */
  dtx += du * fx / tz;
  dty += dv * fy / tz;
  dtz += -du * fx * p->tx / tz2 - dv * fy * p->ty / tz2;
  /* t = R m + t_c */
  gm[0] += V[0] * dtx + V[4] * dty + V[8] * dtz;
  gm[1] += V[1] * dtx + V[5] * dty + V[9] * dtz;
  gm[2] += V[2] * dtx + V[6] * dty + V[10] * dtz;
}

/* Backward of the render over rows y_begin, y_begin + y_step, ... < y_end
 * (the full image for 0, H, 1).  Upstream gradients (any may be NULL):
 * d_rgb[H,W,3], d_depth[H,W], d_sil[H,W], d_sem[H,W,m].  Gradients are
 * ACCUMULATED into g_means[n,3], g_scales[n,3], g_quats[n,4], g_opacity[n],
 * g_rgb[n,3], g_sem_w[n,k].  When sem_detach != 0 the semantic upstream
 * gradient reaches only g_sem_w (Sec. 3.1, semantic loss restricted to the
 * semantic attributes). */
void SFX(orc_render_bwd)(int n, int k, int m, const real *means, const real *scales, const real *quats,
                         const real *opacity, const real *rgb, const int *sem_ids, const real *sem_w,
                         const real *cam, int W, int H, const real *d_rgb, const real *d_depth,
                         const real *d_sil, const real *d_sem, int sem_detach, real *g_means,
                         real *g_scales, real *g_quats, real *g_opacity, real *g_rgb, real *g_sem_w,
                         int y_begin, int y_end, int y_step) {
  const real *unc = NULL;
  SCENE_FROM_ARGS
  view_t vw;
  view_build(&sc, cam, W, H, &vw);
  /* Rows are shared round-robin among the threads; each thread accumulates
   * its pixels' terms per visible Gaussian in a private array: du dv dca dcb
   * dcc dz (2D gradients), r g b, opacity, then k semantic weights.  The
   * arrays are added in thread order at the end, so a given thread count
   * gives the same sums on every run. */
  const int nv = vw.nv, stride = 10 + k;
  int *vis_of = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int g = 0; g < n; ++g) vis_of[g] = -1;
  for (int i = 0; i < nv; ++i) vis_of[vw.order[i]] = i;
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  real *acc_all = (real *)calloc((size_t)nthr * (size_t)(nv > 0 ? nv : 1) * (size_t)stride, sizeof(real));
  const int cap = nv > 0 ? nv : 1;
  if (y_step < 1) y_step = 1;
  if (y_end > H || y_end < 0) y_end = H;
  const int nrows = y_end > y_begin ? (y_end - y_begin + y_step - 1) / y_step : 0;
#pragma omp parallel num_threads(nthr)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    real *A = acc_all + (size_t)t * (size_t)(nv > 0 ? nv : 1) * (size_t)stride;
    contrib_t *list = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)cap);
#pragma omp for schedule(static, 1)
    for (int r = 0; r < nrows; ++r) {
      const int y = y_begin + r * y_step;
      for (int x = 0; x < W; ++x) {
        size_t pid = (size_t)y * W + x;
        pix_t o;
        composite_pixel(&sc, &vw, x, y, NULL, &o, list, cap);
        real dc[3] = {0, 0, 0}, dd = 0, ds = 0;
        if (d_rgb) { dc[0] = d_rgb[3 * pid]; dc[1] = d_rgb[3 * pid + 1]; dc[2] = d_rgb[3 * pid + 2]; }
        if (d_depth) dd = d_depth[pid];
        if (d_sil) ds = d_sil[pid];
        const real *dp = d_sem ? d_sem + pid * m : NULL;
        real acc = 0; /* sum over later contributors of w_j * g_j */
        for (int i = o.n_contrib - 1; i >= 0; --i) {
          const contrib_t *c = &list[i];
          int g = c->gid;
          const proj_t *p = &vw.proj[g];
          real *e = A + (size_t)vis_of[g] * stride;
          real w = c->alpha * c->T;
          real gi = dc[0] * sc.rgb[3 * g] + dc[1] * sc.rgb[3 * g + 1] + dc[2] * sc.rgb[3 * g + 2] +
                    dd * p->tz + ds;
          real gsem = 0;
          for (int j = 0; j < k; ++j) {
            real dpj = dp ? dp[sc.sem_ids[g * k + j]] : 0;
            e[10 + j] += dpj * w;
            gsem += dpj * sc.sem_w[g * k + j];
          }
          if (!sem_detach) gi += gsem;
          for (int ch = 0; ch < 3; ++ch) e[6 + ch] += dc[ch] * w;
          e[5] += dd * w;
          real dalpha = c->T * gi - acc / ((real)1 - c->alpha);
          acc += w * gi;
          if (c->a < ALPHA_MAX) {
            e[9] += dalpha * c->G;
            real dpow = dalpha * c->a;
            real dx = c->dx, dy = c->dy;
            e[2] += dpow * (-(real)0.5 * dx * dx);
            e[3] += dpow * (-dx * dy);
            e[4] += dpow * (-(real)0.5 * dy * dy);
            e[0] += dpow * (-(p->ca * dx + p->cb * dy));
            e[1] += dpow * (-(p->cc * dy + p->cb * dx));
          }
        }
      }
    }
    free(list);
  }
#pragma omp parallel
  {
    real *e = (real *)malloc(sizeof(real) * (size_t)stride);
#pragma omp for schedule(static)
    for (int i = 0; i < nv; ++i) {
      const int g = vw.order[i];
      const proj_t *p = &vw.proj[g];
      for (int q = 0; q < stride; ++q) e[q] = 0;
      for (int t = 0; t < nthr; ++t) {
        const real *src = acc_all + ((size_t)t * (size_t)nv + (size_t)i) * (size_t)stride;
        for (int q = 0; q < stride; ++q) e[q] += src[q];
      }
      for (int ch = 0; ch < 3; ++ch) g_rgb[3 * g + ch] += e[6 + ch];
      g_opacity[g] += e[9];
      for (int j = 0; j < k; ++j) g_sem_w[g * k + j] += e[10 + j];
      project_adjoint(p, scales + 3 * g, cam, e[0], e[1], e[2], e[3], e[4], e[5], g_means + 3 * g,
                      g_scales + 3 * g, g_quats + 4 * g);
    }
    free(e);
  }
  free(acc_all);
  free(vis_of);
  view_free(&vw);
}

/* ------------------------------------------------------------------------ */
/* Candidate-view reductions                                                 */
/* ------------------------------------------------------------------------ */

/* For one view: sumU = sum_p U(p), sumH = sum_p H(p) of the clipped
 * ([0.001, 1]) and renormalised semantic map, N_S = #{p : S(p) = 0}
 * (Eq. 6, Eq. 7 with Eq. 4).  Reductions in double.  out[3] = {sumU, sumH,
 * N_S}; n_flag = number of pixels with a near-threshold decision. */
void SFX(orc_candidate)(int n, int k, int m, const real *means, const real *scales, const real *quats,
                        const real *opacity, const real *rgb, const int *sem_ids, const real *sem_w,
                        const real *unc, const real *cam, int W, int H, double *out, long *n_flag) {
  SCENE_FROM_ARGS
  view_t vw;
  view_build(&sc, cam, W, H, &vw);
  double su = 0, sh = 0, ns = 0;
  long nf = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : su, sh, ns, nf)
  for (int y = 0; y < H; ++y) {
    real *sem = (real *)malloc(sizeof(real) * (size_t)m);
    double *ph = (double *)malloc(sizeof(double) * (size_t)m);
    for (int x = 0; x < W; ++x) {
      memset(sem, 0, sizeof(real) * (size_t)m);
      pix_t o;
      composite_pixel(&sc, &vw, x, y, sem, &o, NULL, 0);
      su += (double)o.unc;
      if ((real)1 - o.T == 0) ns += 1;
      nf += o.flag & 1;
      double z = 0;
      for (int c = 0; c < m; ++c) {
        double v = (double)sem[c];
        ph[c] = v < 0.001 ? 0.001 : (v > 1.0 ? 1.0 : v);
        z += ph[c];
      }
      double h = 0;
      for (int c = 0; c < m; ++c) {
        double q = ph[c] / z;
        h -= q * log(q);
      }
      sh += h;
    }
    free(sem);
    free(ph);
  }
  out[0] = su; out[1] = sh; out[2] = ns;
  if (n_flag) *n_flag = nf;
  view_free(&vw);
}
