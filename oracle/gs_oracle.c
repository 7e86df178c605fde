/*
 * FP64 CPU oracle — TEST INFRASTRUCTURE ONLY (see gs_oracle.h).
 *
 * Plain loops, double precision, no tiling except in orc_render_tiled, which
 * exists only to pin the tile-invariance of the support rule.  Each function
 * cites the passage of the paper it restates; a silent or ambiguous point
 * takes the published 3DGS convention, stated where it is applied (the
 * compositing constants below, for instance).
 */
#include "gs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Compositing constants: the published 3DGS choices, which the paper takes
 * over through its rasterizer (Sec. 3.3 "Implementation"). */
#define ALPHA_MIN (1.0 / 255.0) /* a splat contributes iff alpha >= 1/255  */
#define ALPHA_MAX 0.99          /* alpha is clamped at 0.99                */
#define T_MIN 1e-4              /* stop before T' would fall below 1e-4   */
#define DILATION 0.3            /* screen-space covariance dilation (px^2) */
#define GUARD 1.3               /* guard band of the EWA Jacobian           */
#define RECT_MARGIN (1.0 / 64.0) /* px around the support's bounding box      */

/* ------------------------------------------------------------------------ */
/* small dense linear algebra                                               */

static void m3_mul(const double* A, const double* B, double* C) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
      C[3 * r + c] = s;
    }
}

static void m3_transpose(const double* A, double* B) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) B[3 * c + r] = A[3 * r + c];
}

static void m3_vec(const double* A, const double* x, double* y) {
  for (int r = 0; r < 3; ++r)
    y[r] = A[3 * r] * x[0] + A[3 * r + 1] * x[1] + A[3 * r + 2] * x[2];
}

static void m3_tvec(const double* A, const double* x, double* y) {
  for (int c = 0; c < 3; ++c)
    y[c] = A[c] * x[0] + A[3 + c] * x[1] + A[6 + c] * x[2];
}

static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

static void skew3(const double* w, double* S) {
  S[0] = 0.0;   S[1] = -w[2]; S[2] = w[1];
  S[3] = w[2];  S[4] = 0.0;   S[5] = -w[0];
  S[6] = -w[1]; S[7] = w[0];  S[8] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* real spherical harmonics, degree <= 3                                    */
/*
 * Sec. 3.3 "Implementation" states SH colour up to degree 3 without fixing a
 * basis.  Reading: the real SH basis in the coefficient order and sign
 * convention of the original 3DGS renderer.  Each normalisation constant is
 * its textbook closed form; the basis is pinned by an orthonormality test.
 * Y is [K], dY is [K][3] = d Y / d(x,y,z) of the polynomial form.
 */
int orc_sh_eval(int degree, const double d[3], double* Y, double* dY) {
  if (degree < 0 || degree > 3) return -1;
  const double pi = M_PI;
  const double c0 = 0.5 * sqrt(1.0 / pi);
  const double c1 = sqrt(3.0 / (4.0 * pi));
  const double c2a = 0.5 * sqrt(15.0 / pi);
  const double c2b = 0.25 * sqrt(5.0 / pi);
  const double c2c = 0.25 * sqrt(15.0 / pi);
  const double c3a = 0.25 * sqrt(35.0 / (2.0 * pi));
  const double c3b = 0.5 * sqrt(105.0 / pi);
  const double c3c = 0.25 * sqrt(21.0 / (2.0 * pi));
  const double c3d = 0.25 * sqrt(7.0 / pi);
  const double c3e = 0.25 * sqrt(105.0 / pi);
  const double x = d[0], y = d[1], z = d[2];
  const int K = (degree + 1) * (degree + 1);
  double g[16][3];
  double v[16];
  memset(g, 0, sizeof(g));
  v[0] = c0;
  if (degree >= 1) {
    v[1] = -c1 * y; g[1][1] = -c1;
    v[2] = c1 * z;  g[2][2] = c1;
    v[3] = -c1 * x; g[3][0] = -c1;
  }
  if (degree >= 2) {
    v[4] = c2a * x * y;
    g[4][0] = c2a * y; g[4][1] = c2a * x;
    v[5] = -c2a * y * z;
    g[5][1] = -c2a * z; g[5][2] = -c2a * y;
    v[6] = c2b * (2.0 * z * z - x * x - y * y);
    g[6][0] = -2.0 * c2b * x; g[6][1] = -2.0 * c2b * y; g[6][2] = 4.0 * c2b * z;
    v[7] = -c2a * x * z;
    g[7][0] = -c2a * z; g[7][2] = -c2a * x;
    v[8] = c2c * (x * x - y * y);
    g[8][0] = 2.0 * c2c * x; g[8][1] = -2.0 * c2c * y;
  }
  if (degree >= 3) {
    v[9] = -c3a * y * (3.0 * x * x - y * y);
    g[9][0] = -c3a * 6.0 * x * y;
    g[9][1] = -c3a * (3.0 * x * x - 3.0 * y * y);
    v[10] = c3b * x * y * z;
    g[10][0] = c3b * y * z; g[10][1] = c3b * x * z; g[10][2] = c3b * x * y;
    v[11] = -c3c * y * (4.0 * z * z - x * x - y * y);
    g[11][0] = c3c * 2.0 * x * y;
    g[11][1] = -c3c * (4.0 * z * z - x * x - 3.0 * y * y);
    g[11][2] = -c3c * 8.0 * y * z;
    v[12] = c3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    g[12][0] = -c3d * 6.0 * x * z;
    g[12][1] = -c3d * 6.0 * y * z;
    g[12][2] = c3d * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    v[13] = -c3c * x * (4.0 * z * z - x * x - y * y);
    g[13][0] = -c3c * (4.0 * z * z - 3.0 * x * x - y * y);
    g[13][1] = c3c * 2.0 * x * y;
    g[13][2] = -c3c * 8.0 * x * z;
    v[14] = c3e * z * (x * x - y * y);
    g[14][0] = c3e * 2.0 * x * z; g[14][1] = -c3e * 2.0 * y * z;
    g[14][2] = c3e * (x * x - y * y);
    v[15] = -c3a * x * (x * x - 3.0 * y * y);
    g[15][0] = -c3a * (3.0 * x * x - 3.0 * y * y);
    g[15][1] = c3a * 6.0 * x * y;
  }
  for (int k = 0; k < K; ++k) {
    if (Y) Y[k] = v[k];
    if (dY)
      for (int i = 0; i < 3; ++i) dY[3 * k + i] = g[k][i];
  }
  return K;
}

/* ------------------------------------------------------------------------ */
/* projection of one Gaussian into one camera                               */

typedef struct proj_state {
  int visible;
  double s[3], qn[4], qnorm, Rg[9], M[9], Sigma[9];
  double xc[3], Sc[9];
  double ux, uy, tx, ty;
  int clamp_x, clamp_y;
  double J[6];     /* 2x3 row-major */
  double S2[4];    /* 2x2 row-major, includes the dilation */
  double det, conic[3];
  double m2[2];
  double o;
  double campos[3], dvec[3], dnorm, dir[3];
  double color_raw[3], color[3];
  double bound[4];
  double px[4];
} proj_state;

/* Unit quaternion (w,x,y,z) to rotation matrix (row-major). */
static void quat_to_rot(const double* q, double* R) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - w * z);
  R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);
  R[7] = 2.0 * (y * z + w * x);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/*
 * Forward projection (rasterizer of Sec. 3.3; pi of Sec. 3.2 for the mean):
 * activations, world covariance, camera transform, near/far cull, EWA 2-D
 * covariance with guard band and dilation, conic, mean2d, opacity-aware
 * conservative pixel rectangle, SH colour.
 */
static void project_one(const orc_scene* sc, int j, const orc_camera* cam,
                        proj_state* P) {
  memset(P, 0, sizeof(*P));
  const double* mu = sc->mean + 3 * j;
  const double* W = cam->R;
  m3_vec(W, mu, P->xc);
  for (int i = 0; i < 3; ++i) P->xc[i] += cam->t[i];
  const double z = P->xc[2];
  if (!(z >= cam->near_plane && z <= cam->far_plane)) return;

  const double* ls = sc->log_scale + 3 * j;
  for (int i = 0; i < 3; ++i) P->s[i] = exp(ls[i]);
  const double* q = sc->quat + 4 * j;
  P->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(P->qnorm > 0.0)) return;
  for (int i = 0; i < 4; ++i) P->qn[i] = q[i] / P->qnorm;
  quat_to_rot(P->qn, P->Rg);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) P->M[3 * r + c] = P->Rg[3 * r + c] * P->s[c];
  double Mt[9], Wt[9], tmp[9];
  m3_transpose(P->M, Mt);
  m3_mul(P->M, Mt, P->Sigma);
  m3_transpose(W, Wt);
  m3_mul(W, P->Sigma, tmp);
  m3_mul(tmp, Wt, P->Sc);

  const double fx = cam->fx, fy = cam->fy;
  P->ux = P->xc[0] / z;
  P->uy = P->xc[1] / z;
  const double limx = GUARD * 0.5 * cam->width / fx;
  const double limy = GUARD * 0.5 * cam->height / fy;
  P->tx = P->ux;
  P->ty = P->uy;
  if (P->tx < -limx) { P->tx = -limx; P->clamp_x = 1; }
  if (P->tx > limx) { P->tx = limx; P->clamp_x = 1; }
  if (P->ty < -limy) { P->ty = -limy; P->clamp_y = 1; }
  if (P->ty > limy) { P->ty = limy; P->clamp_y = 1; }
  double* J = P->J;
  J[0] = fx / z; J[1] = 0.0; J[2] = -fx * P->tx / z;
  J[3] = 0.0; J[4] = fy / z; J[5] = -fy * P->ty / z;
  /* S2 = J Sc J^T + DILATION I */
  double JS[6];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += J[3 * r + k] * P->Sc[3 * k + c];
      JS[3 * r + c] = s;
    }
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += JS[3 * r + k] * J[3 * c + k];
      P->S2[2 * r + c] = s;
    }
  P->S2[0] += DILATION;
  P->S2[3] += DILATION;
  P->det = P->S2[0] * P->S2[3] - P->S2[1] * P->S2[2];
  if (!(P->det > 0.0)) return;
  P->conic[0] = P->S2[3] / P->det;
  P->conic[1] = -P->S2[1] / P->det;
  P->conic[2] = P->S2[0] / P->det;
  P->m2[0] = fx * P->ux + cam->cx;
  P->m2[1] = fy * P->uy + cam->cy;

  P->o = 1.0 / (1.0 + exp(-sc->opacity_logit[j]));
  if (P->o < ALPHA_MIN) return;
  /* alpha >= 1/255 <=> q <= Q; the ellipse q <= Q has half-widths
   * sqrt(Q S2_xx), sqrt(Q S2_yy).  Pixel u is covered iff its centre u+0.5
   * lies within; RECT_MARGIN (1/64 px, about a hundred times the float
   * rounding of the bounds at these image sizes) on each side keeps a float
   * evaluation of the rectangle conservative. */
  const double Q = 2.0 * log(255.0 * P->o);
  const double rx = sqrt(Q * P->S2[0]);
  const double ry = sqrt(Q * P->S2[3]);
  P->bound[0] = P->m2[0] - rx - 0.5;
  P->bound[1] = P->m2[1] - ry - 0.5;
  P->bound[2] = P->m2[0] + rx - 0.5;
  P->bound[3] = P->m2[1] + ry - 0.5;
  double x0 = ceil(P->bound[0] - RECT_MARGIN), y0 = ceil(P->bound[1] - RECT_MARGIN);
  double x1 = floor(P->bound[2] + RECT_MARGIN), y1 = floor(P->bound[3] + RECT_MARGIN);
  if (x0 < 0.0) x0 = 0.0;
  if (y0 < 0.0) y0 = 0.0;
  if (x1 > cam->width - 1.0) x1 = cam->width - 1.0;
  if (y1 > cam->height - 1.0) y1 = cam->height - 1.0;
  if (x0 > x1 || y0 > y1) return;
  P->px[0] = x0; P->px[1] = y0; P->px[2] = x1; P->px[3] = y1;

  /* view-dependent colour: dir from the camera centre c = -R^T t */
  m3_tvec(W, cam->t, P->campos);
  for (int i = 0; i < 3; ++i) P->campos[i] = -P->campos[i];
  for (int i = 0; i < 3; ++i) P->dvec[i] = mu[i] - P->campos[i];
  P->dnorm = sqrt(P->dvec[0] * P->dvec[0] + P->dvec[1] * P->dvec[1] +
                  P->dvec[2] * P->dvec[2]);
  for (int i = 0; i < 3; ++i) P->dir[i] = P->dvec[i] / P->dnorm;
  const int K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
  double Y[16];
  orc_sh_eval(sc->sh_degree, P->dir, Y, NULL);
  const double* sh = sc->sh + (size_t)j * K * 3;
  for (int ch = 0; ch < 3; ++ch) {
    double v = 0.5;
    for (int k = 0; k < K; ++k) v += sh[3 * k + ch] * Y[k];
    P->color_raw[ch] = v;
    P->color[ch] = v < 0.0 ? 0.0 : v;
  }
  P->visible = 1;
}

int orc_project(const orc_scene* sc, const orc_camera* cam, double* out) {
  proj_state P;
  for (int j = 0; j < sc->n; ++j) {
    project_one(sc, j, cam, &P);
    double* o = out + (size_t)j * ORC_P_FIELDS;
    memset(o, 0, sizeof(double) * ORC_P_FIELDS);
    o[ORC_P_VISIBLE] = P.visible;
    o[ORC_P_DEPTH] = P.xc[2];
    o[ORC_P_XC] = P.xc[0];
    o[ORC_P_YC] = P.xc[1];
    o[ORC_P_MX] = P.m2[0];
    o[ORC_P_MY] = P.m2[1];
    o[ORC_P_COV_XX] = P.S2[0];
    o[ORC_P_COV_XY] = P.S2[1];
    o[ORC_P_COV_YY] = P.S2[3];
    o[ORC_P_CON_A] = P.conic[0];
    o[ORC_P_CON_B] = P.conic[1];
    o[ORC_P_CON_C] = P.conic[2];
    o[ORC_P_OPACITY] = P.o;
    for (int ch = 0; ch < 3; ++ch) o[ORC_P_R + ch] = P.color[ch];
    for (int i = 0; i < 4; ++i) o[ORC_P_BOUND_X0 + i] = P.bound[i];
    for (int i = 0; i < 4; ++i) o[ORC_P_PX_X0 + i] = P.px[i];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* depth ordering                                                           */

typedef struct order_item {
  double depth;
  int j;
} order_item;

static int cmp_order(const void* a, const void* b) {
  const order_item* x = (const order_item*)a;
  const order_item* y = (const order_item*)b;
  if (x->depth < y->depth) return -1;
  if (x->depth > y->depth) return 1;
  return (x->j > y->j) - (x->j < y->j);
}

/* Visible Gaussians of a view, sorted front to back by (camera depth z,
 * index j).  Reading: depth is camera-space z; ties broken by j. */
static int visible_order(const orc_scene* sc, const orc_camera* cam,
                         proj_state** states_out, int** order_out) {
  proj_state* st = (proj_state*)malloc(sizeof(proj_state) * (size_t)(sc->n > 0 ? sc->n : 1));
  order_item* items = (order_item*)malloc(sizeof(order_item) * (size_t)(sc->n > 0 ? sc->n : 1));
  int nv = 0;
  for (int j = 0; j < sc->n; ++j) {
    project_one(sc, j, cam, &st[j]);
    if (st[j].visible) {
      items[nv].depth = st[j].xc[2];
      items[nv].j = j;
      ++nv;
    }
  }
  qsort(items, (size_t)nv, sizeof(order_item), cmp_order);
  int* order = (int*)malloc(sizeof(int) * (size_t)(nv > 0 ? nv : 1));
  for (int k = 0; k < nv; ++k) order[k] = items[k].j;
  free(items);
  *states_out = st;
  *order_out = order;
  return nv;
}

/* ------------------------------------------------------------------------ */
/* per-pixel compositing (front to back)                                    */

typedef struct contrib {
  int j;
  double alpha, G, og, dx, dy, T_before;
} contrib;

/*
 * Composite one pixel over the ordered list (Algorithm 1, "Rasterize").
 * For each splat: alpha = min(0.99, o exp(-q/2)); skip if alpha < 1/255;
 * T' = T (1 - alpha); stop before adding it if T' < 1e-4; else
 * C += c alpha T, T = T'.  Finally C += T bg.
 */
static void composite_pixel(const proj_state* st, const int* order, int nv,
                            double u, double v, const double* bg,
                            double eps, double* C, double* T_out,
                            int* last, int* nadd, int* knife, int64_t* npairs,
                            contrib* rec) {
  double T = 1.0;
  C[0] = C[1] = C[2] = 0.0;
  int n = 0, lastj = -1, flags = 0;
  double prev_depth = -1.0;
  const double px = u + 0.5, py = v + 0.5;
  int64_t pairs = 0;
  for (int k = 0; k < nv; ++k) {
    const proj_state* P = &st[order[k]];
    const double dx = px - P->m2[0];
    const double dy = py - P->m2[1];
    const double q = P->conic[0] * dx * dx + 2.0 * P->conic[1] * dx * dy +
                     P->conic[2] * dy * dy;
    const double G = exp(-0.5 * q);
    const double og = P->o * G;
    const double alpha = og < ALPHA_MAX ? og : ALPHA_MAX;
    ++pairs;
    if (fabs(og - ALPHA_MIN) <= eps * ALPHA_MIN) flags |= ORC_KNIFE_ALPHA_MIN;
    if (alpha < ALPHA_MIN) continue;
    if (fabs(og - ALPHA_MAX) <= eps * ALPHA_MAX) flags |= ORC_KNIFE_ALPHA_MAX;
    const double Tn = T * (1.0 - alpha);
    if (fabs(Tn - T_MIN) <= eps * T_MIN) flags |= ORC_KNIFE_T_MIN;
    if (Tn < T_MIN) break;
    if (prev_depth >= 0.0 && fabs(P->xc[2] - prev_depth) <= 1e-6 * P->xc[2])
      flags |= ORC_KNIFE_DEPTH;
    prev_depth = P->xc[2];
    if (rec) {
      rec[n].j = order[k];
      rec[n].alpha = alpha;
      rec[n].G = G;
      rec[n].og = og;
      rec[n].dx = dx;
      rec[n].dy = dy;
      rec[n].T_before = T;
    }
    for (int ch = 0; ch < 3; ++ch) C[ch] += P->color[ch] * alpha * T;
    T = Tn;
    lastj = order[k];
    ++n;
  }
  for (int ch = 0; ch < 3; ++ch) C[ch] += T * bg[ch];
  *T_out = T;
  if (last) *last = lastj;
  if (nadd) *nadd = n;
  if (knife) *knife = flags;
  if (npairs) *npairs += pairs;
}

int orc_render(const orc_scene* sc, const orc_camera* cam, const double bg[3],
               int64_t npix, const int32_t* pix, double knife_eps,
               double* image, double* T_final, int32_t* last_id,
               int32_t* n_added, int32_t* knife, int64_t* n_pairs) {
  proj_state* st;
  int* order;
  const int nv = visible_order(sc, cam, &st, &order);
  const int64_t total = pix ? npix : (int64_t)cam->width * cam->height;
  int64_t pairs = 0;
  for (int64_t p = 0; p < total; ++p) {
    int u, v;
    if (pix) { u = pix[2 * p]; v = pix[2 * p + 1]; }
    else { u = (int)(p % cam->width); v = (int)(p / cam->width); }
    double C[3], T;
    int last, nadd, fl;
    composite_pixel(st, order, nv, u, v, bg, knife_eps, C, &T, &last, &nadd,
                    &fl, &pairs, NULL);
    for (int ch = 0; ch < 3; ++ch) image[3 * p + ch] = C[ch];
    if (T_final) T_final[p] = T;
    if (last_id) last_id[p] = last;
    if (n_added) n_added[p] = nadd;
    if (knife) knife[p] = fl;
  }
  if (n_pairs) *n_pairs = pairs;
  free(st);
  free(order);
  return 0;
}

/*
 * Tiled variant, used only to pin that the opacity-aware rectangle is
 * conservative: every tile composites the Gaussians whose pixel rectangle
 * meets it, in the same (depth, index) order; the image must equal the
 * untiled one exactly.
 */
int orc_render_tiled(const orc_scene* sc, const orc_camera* cam,
                     const double bg[3], int tile, double* image,
                     double* T_final) {
  if (tile <= 0) return -1;
  proj_state* st;
  int* order;
  const int nv = visible_order(sc, cam, &st, &order);
  int* list = (int*)malloc(sizeof(int) * (size_t)(nv > 0 ? nv : 1));
  const int tx_n = (cam->width + tile - 1) / tile;
  const int ty_n = (cam->height + tile - 1) / tile;
  for (int ty = 0; ty < ty_n; ++ty)
    for (int tx = 0; tx < tx_n; ++tx) {
      int nl = 0;
      for (int k = 0; k < nv; ++k) {
        const proj_state* P = &st[order[k]];
        const int gx0 = (int)P->px[0] / tile, gy0 = (int)P->px[1] / tile;
        const int gx1 = (int)P->px[2] / tile, gy1 = (int)P->px[3] / tile;
        if (tx >= gx0 && tx <= gx1 && ty >= gy0 && ty <= gy1) list[nl++] = order[k];
      }
      for (int v = ty * tile; v < (ty + 1) * tile && v < cam->height; ++v)
        for (int u = tx * tile; u < (tx + 1) * tile && u < cam->width; ++u) {
          double C[3], T;
          composite_pixel(st, list, nl, u, v, bg, 0.0, C, &T, NULL, NULL, NULL,
                          NULL, NULL);
          const int64_t p = (int64_t)v * cam->width + u;
          for (int ch = 0; ch < 3; ++ch) image[3 * p + ch] = C[ch];
          if (T_final) T_final[p] = T;
        }
    }
  free(list);
  free(st);
  free(order);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* backward                                                                 */

/*
 * Reverse of project_one for one (Gaussian, camera) pair, given the
 * gradient of the loss w.r.t. the screen-space record
 * v2d = (mean2d x, y, conic a, b, c, opacity, colour r, g, b), where the
 * conic enters q = a dx^2 + 2 b dx dy + c dy^2.  Accumulates into the raw
 * parameter gradients and into the camera's G_W (dL/dR, 3x3) and v_t.
 * Clamps (alpha at 0.99 is handled by the caller; colour at 0, guard band)
 * pass zero gradient.
 */
static void project_bwd(const orc_scene* sc, int j, const orc_camera* cam,
                        const proj_state* P, const double* v2d,
                        double* v_mean, double* v_log_scale, double* v_quat,
                        double* v_opl, double* v_sh, double* GW, double* vt) {
  const double* mu = sc->mean + 3 * j;
  const double* W = cam->R;
  const double fx = cam->fx, fy = cam->fy;
  const double z = P->xc[2];
  const int K = (sc->sh_degree + 1) * (sc->sh_degree + 1);

  /* colour */
  double vc[3];
  for (int ch = 0; ch < 3; ++ch) vc[ch] = P->color_raw[ch] < 0.0 ? 0.0 : v2d[6 + ch];
  double Y[16], dY[48];
  orc_sh_eval(sc->sh_degree, P->dir, Y, dY);
  const double* sh = sc->sh + (size_t)j * K * 3;
  double v_dir[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < K; ++k)
    for (int ch = 0; ch < 3; ++ch) {
      v_sh[(size_t)j * K * 3 + 3 * k + ch] += Y[k] * vc[ch];
      for (int i = 0; i < 3; ++i) v_dir[i] += sh[3 * k + ch] * vc[ch] * dY[3 * k + i];
    }
  const double dd = v_dir[0] * P->dir[0] + v_dir[1] * P->dir[1] + v_dir[2] * P->dir[2];
  double v_dvec[3], v_campos[3];
  for (int i = 0; i < 3; ++i) {
    v_dvec[i] = (v_dir[i] - dd * P->dir[i]) / P->dnorm;
    v_mean[3 * j + i] += v_dvec[i];
    v_campos[i] = -v_dvec[i];
  }

  /* opacity */
  v_opl[j] += v2d[5] * P->o * (1.0 - P->o);

  /* conic = inverse(S2):  dL/dS2 = -Q GQ Q with GQ the symmetric gradient */
  const double Qm[4] = {P->conic[0], P->conic[1], P->conic[1], P->conic[2]};
  const double GQ[4] = {v2d[2], 0.5 * v2d[3], 0.5 * v2d[3], v2d[4]};
  double T1[4], GS2[4];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c)
      T1[2 * r + c] = Qm[2 * r] * GQ[c] + Qm[2 * r + 1] * GQ[2 + c];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c)
      GS2[2 * r + c] = -(T1[2 * r] * Qm[c] + T1[2 * r + 1] * Qm[2 + c]);

  /* S2 = J Sc J^T (+ dilation):  GSc = J^T GS2 J,  GJ = 2 GS2 J Sc */
  const double* J = P->J;
  double GSc[9], GJ[6], GJ1[6];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) s += J[3 * r + a] * GS2[2 * r + c] * J[3 * c + b];
      GSc[3 * a + b] = s;
    }
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 2; ++k) s += GS2[2 * r + k] * J[3 * k + c];
      GJ1[3 * r + c] = s;
    }
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += GJ1[3 * r + k] * P->Sc[3 * k + c];
      GJ[3 * r + c] = 2.0 * s;
    }

  /* Sc = W Sigma W^T:  GSigma = W^T GSc W,  GW += 2 GSc W Sigma */
  double Wt[9], tmp[9], tmp2[9], GSigma[9];
  m3_transpose(W, Wt);
  m3_mul(Wt, GSc, tmp);
  m3_mul(tmp, W, GSigma);
  m3_mul(GSc, W, tmp);
  m3_mul(tmp, P->Sigma, tmp2);
  for (int i = 0; i < 9; ++i) GW[i] += 2.0 * tmp2[i];

  /* Sigma = M M^T, M = Rg diag(s) */
  double GM[9];
  m3_mul(GSigma, P->M, GM);
  for (int i = 0; i < 9; ++i) GM[i] *= 2.0;
  double GR[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) GR[3 * r + c] = GM[3 * r + c] * P->s[c];
  for (int c = 0; c < 3; ++c) {
    double gs = 0.0;
    for (int r = 0; r < 3; ++r) gs += GM[3 * r + c] * P->Rg[3 * r + c];
    v_log_scale[3 * j + c] += gs * P->s[c];
  }
  /* Rg(qn): partial derivatives of each entry w.r.t. (w,x,y,z) */
  {
    const double w = P->qn[0], x = P->qn[1], y = P->qn[2], zq = P->qn[3];
    const double d[9][4] = {
        {0.0, 0.0, -4.0 * y, -4.0 * zq},
        {-2.0 * zq, 2.0 * y, 2.0 * x, -2.0 * w},
        {2.0 * y, 2.0 * zq, 2.0 * w, 2.0 * x},
        {2.0 * zq, 2.0 * y, 2.0 * x, 2.0 * w},
        {0.0, -4.0 * x, 0.0, -4.0 * zq},
        {-2.0 * x, -2.0 * w, 2.0 * zq, 2.0 * y},
        {-2.0 * y, 2.0 * zq, -2.0 * w, 2.0 * x},
        {2.0 * x, 2.0 * w, 2.0 * zq, 2.0 * y},
        {0.0, -4.0 * x, -4.0 * y, 0.0}};
    double vqn[4] = {0.0, 0.0, 0.0, 0.0};
    for (int e = 0; e < 9; ++e)
      for (int i = 0; i < 4; ++i) vqn[i] += GR[e] * d[e][i];
    double dot = 0.0;
    for (int i = 0; i < 4; ++i) dot += vqn[i] * P->qn[i];
    for (int i = 0; i < 4; ++i) v_quat[4 * j + i] += (vqn[i] - dot * P->qn[i]) / P->qnorm;
  }

  /* J(x_c) with guard-band clamp t = clamp(x/z) */
  double vxc[3] = {0.0, 0.0, 0.0};
  const double dJ02dx = P->clamp_x ? 0.0 : -fx / (z * z);
  const double dJ12dy = P->clamp_y ? 0.0 : -fy / (z * z);
  const double dJ02dz = fx * P->tx / (z * z) + (P->clamp_x ? 0.0 : fx * P->xc[0] / (z * z * z));
  const double dJ12dz = fy * P->ty / (z * z) + (P->clamp_y ? 0.0 : fy * P->xc[1] / (z * z * z));
  vxc[0] += GJ[2] * dJ02dx;
  vxc[1] += GJ[5] * dJ12dy;
  vxc[2] += GJ[0] * (-fx / (z * z)) + GJ[4] * (-fy / (z * z)) + GJ[2] * dJ02dz +
            GJ[5] * dJ12dz;

  /* mean2d = (fx x/z + cx, fy y/z + cy) */
  vxc[0] += v2d[0] * fx / z;
  vxc[1] += v2d[1] * fy / z;
  vxc[2] -= (v2d[0] * fx * P->xc[0] + v2d[1] * fy * P->xc[1]) / (z * z);

  /* x_c = W mu + t */
  double vmu[3];
  m3_tvec(W, vxc, vmu);
  for (int i = 0; i < 3; ++i) v_mean[3 * j + i] += vmu[i];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) GW[3 * r + c] += vxc[r] * mu[c];
  for (int i = 0; i < 3; ++i) vt[i] += vxc[i];

  /* camera centre c = -W^T t */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) GW[3 * r + c] += -cam->t[r] * v_campos[c];
  double Wv[3];
  m3_vec(W, v_campos, Wv);
  for (int i = 0; i < 3; ++i) vt[i] -= Wv[i];
}

/* Left-perturbation tangent from the gradients w.r.t. (R, t):
 * g_rho = dL/dt,  g_phi = vee(G_W R^T) + t x dL/dt. */
static void tangent_from_GW(const orc_camera* cam, const double* GW,
                            const double* vt, double* g) {
  double Wt[9], A[9], tv[3];
  m3_transpose(cam->R, Wt);
  m3_mul(GW, Wt, A);
  cross3(cam->t, vt, tv);
  g[0] = vt[0];
  g[1] = vt[1];
  g[2] = vt[2];
  g[3] = (A[7] - A[5]) + tv[0];
  g[4] = (A[2] - A[6]) + tv[1];
  g[5] = (A[3] - A[1]) + tv[2];
}

/*
 * Backward of orc_render for a given dL/dimage (Eq. 5's photometric term
 * enters only through v_image).  Exact derivative of the forward above:
 * dC/dc_k = alpha_k T_k; dC/dalpha_k = c_k T_k - S_k / (1 - alpha_k) with
 * S_k the colour composited behind k (incl. T_final bg); then through
 * alpha = o exp(-q/2) (zero above the 0.99 clamp) and project_bwd.
 * All outputs accumulate (+=).  v2d, if not NULL, receives the per-Gaussian
 * screen-space gradients [n][9] (accumulated); v_tangent_abs, if not NULL,
 * the sum over Gaussians of the absolute value of each one's pose-tangent
 * contribution (the scale of the cancelling pose sum).
 */
int orc_render_bwd(const orc_scene* sc, const orc_camera* cam,
                   const double bg[3], int64_t npix, const int32_t* pix,
                   const double* v_image, double* v_mean, double* v_log_scale,
                   double* v_quat, double* v_opacity_logit, double* v_sh,
                   double* v_tangent, double* v_tangent_abs, double* v2d_out) {
  proj_state* st;
  int* order;
  const int nv = visible_order(sc, cam, &st, &order);
  double* v2d = (double*)calloc((size_t)(sc->n > 0 ? sc->n : 1) * 9, sizeof(double));
  contrib* rec = (contrib*)malloc(sizeof(contrib) * (size_t)(nv > 0 ? nv : 1));
  const int64_t total = pix ? npix : (int64_t)cam->width * cam->height;
  for (int64_t p = 0; p < total; ++p) {
    int u, v;
    if (pix) { u = pix[2 * p]; v = pix[2 * p + 1]; }
    else { u = (int)(p % cam->width); v = (int)(p / cam->width); }
    const double* vC = v_image + 3 * p;
    if (vC[0] == 0.0 && vC[1] == 0.0 && vC[2] == 0.0) continue;
    double C[3], T;
    int nadd;
    composite_pixel(st, order, nv, u, v, bg, 0.0, C, &T, NULL, &nadd, NULL,
                    NULL, rec);
    double S[3];
    for (int ch = 0; ch < 3; ++ch) S[ch] = T * bg[ch];
    for (int k = nadd - 1; k >= 0; --k) {
      const contrib* r = &rec[k];
      const proj_state* P = &st[r->j];
      const double Tk = r->T_before;
      double va = 0.0;
      double* g = v2d + 9 * (size_t)r->j;
      for (int ch = 0; ch < 3; ++ch) {
        g[6 + ch] += r->alpha * Tk * vC[ch];
        va += vC[ch] * (P->color[ch] * Tk - S[ch] / (1.0 - r->alpha));
        S[ch] += P->color[ch] * r->alpha * Tk;
      }
      if (r->og < ALPHA_MAX) {
        const double vq = -0.5 * r->alpha * va; /* dalpha/dq = -alpha/2 */
        g[5] += va * r->G;                      /* dalpha/do = G        */
        const double a = P->conic[0], b = P->conic[1], c = P->conic[2];
        /* q = a dx^2 + 2 b dx dy + c dy^2, d = pixel - mean2d */
        g[0] += vq * (-2.0) * (a * r->dx + b * r->dy);
        g[1] += vq * (-2.0) * (b * r->dx + c * r->dy);
        g[2] += vq * r->dx * r->dx;
        g[3] += vq * 2.0 * r->dx * r->dy;
        g[4] += vq * r->dy * r->dy;
      }
    }
  }
  double GW[9] = {0}, vt[3] = {0};
  for (int j = 0; j < sc->n; ++j) {
    if (!st[j].visible) continue;
    const double* g = v2d + 9 * (size_t)j;
    int nz = 0;
    for (int i = 0; i < 9; ++i) nz |= (g[i] != 0.0);
    if (!nz) continue;
    double GWj[9] = {0}, vtj[3] = {0};
    project_bwd(sc, j, cam, &st[j], g, v_mean, v_log_scale, v_quat,
                v_opacity_logit, v_sh, GWj, vtj);
    for (int i = 0; i < 9; ++i) GW[i] += GWj[i];
    for (int i = 0; i < 3; ++i) vt[i] += vtj[i];
    if (v_tangent_abs) {
      double gj[6];
      tangent_from_GW(cam, GWj, vtj, gj);
      for (int i = 0; i < 6; ++i) v_tangent_abs[i] += fabs(gj[i]);
    }
  }
  if (v_tangent) {
    double gt[6];
    tangent_from_GW(cam, GW, vt, gt);
    for (int i = 0; i < 6; ++i) v_tangent[i] += gt[i];
  }
  if (v2d_out)
    for (size_t i = 0; i < (size_t)sc->n * 9; ++i) v2d_out[i] += v2d[i];
  free(v2d);
  free(rec);
  free(st);
  free(order);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* feature-track reprojection term (Eq. 6)                                  */

/*
 * For each observation (k, i, x): X_c = R_i X_k + t_i, masked (and counted)
 * if Z_c <= near; u = pi_i(X_k) = (fx X/Z + cx, fy Y/Z + cy); r = u - x;
 * s = |r|^2; rho(s) = s if s <= delta^2 else 2 delta sqrt(s) - delta^2.
 * loss += rho (unweighted, Eq. 6); gradients are those of weight * rho and
 * accumulate into grad_X [n_points][3] and the pose tangents [n_cams][6].
 * tangent_abs (may be NULL) accumulates the absolute value of every
 * observation's tangent contribution: the scale against which the
 * cancelling pose sum is compared.
 */
int orc_track(int32_t n_points, const double* X, int64_t n_obs,
              const int32_t* obs_point, const int32_t* obs_cam,
              const double* obs_xy, int32_t n_cams, const orc_camera* cams,
              double delta, double weight, double* loss, double* grad_X,
              double* tangent, double* tangent_abs, int64_t* n_masked) {
  double L = 0.0;
  int64_t masked = 0;
  for (int64_t o = 0; o < n_obs; ++o) {
    const int k = obs_point[o], i = obs_cam[o];
    if (k < 0 || k >= n_points || i < 0 || i >= n_cams) return -1;
    const orc_camera* cam = &cams[i];
    double Xc[3];
    m3_vec(cam->R, X + 3 * k, Xc);
    for (int a = 0; a < 3; ++a) Xc[a] += cam->t[a];
    const double Z = Xc[2];
    if (Z <= cam->near_plane) { ++masked; continue; }
    const double u = cam->fx * Xc[0] / Z + cam->cx;
    const double v = cam->fy * Xc[1] / Z + cam->cy;
    const double rx = u - obs_xy[2 * o], ry = v - obs_xy[2 * o + 1];
    const double s = rx * rx + ry * ry;
    double rho, drho;
    if (s <= delta * delta) { rho = s; drho = 1.0; }
    else { const double rs = sqrt(s); rho = 2.0 * delta * rs - delta * delta; drho = delta / rs; }
    L += rho;
    const double vu = weight * 2.0 * rx * drho;
    const double vv = weight * 2.0 * ry * drho;
    double vXc[3];
    vXc[0] = vu * cam->fx / Z;
    vXc[1] = vv * cam->fy / Z;
    vXc[2] = -(vu * cam->fx * Xc[0] + vv * cam->fy * Xc[1]) / (Z * Z);
    double g[3];
    m3_tvec(cam->R, vXc, g);
    for (int a = 0; a < 3; ++a) grad_X[3 * k + a] += g[a];
    double cr[3];
    cross3(Xc, vXc, cr);
    for (int a = 0; a < 3; ++a) {
      tangent[6 * i + a] += vXc[a];
      tangent[6 * i + 3 + a] += cr[a];
      if (tangent_abs) {
        tangent_abs[6 * i + a] += fabs(vXc[a]);
        tangent_abs[6 * i + 3 + a] += fabs(cr[a]);
      }
    }
  }
  if (loss) *loss += L;
  if (n_masked) *n_masked += masked;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* SE(3) (Algorithm 1: T_i = T_i^(0) (+) dT_i, read as Exp(xi) T0)         */

/* Coefficients of the SO(3)/SE(3) series; Taylor forms near 0. */
static void so3_coeffs(double th, double* A, double* B, double* C) {
  if (th < 1e-4) {
    const double t2 = th * th;
    *A = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
    *B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
    *C = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
  } else {
    *A = sin(th) / th;
    *B = (1.0 - cos(th)) / (th * th);
    *C = (th - sin(th)) / (th * th * th);
  }
}

/* xi = (rho, phi): R = I + A Phi + B Phi^2, V = I + B Phi + C Phi^2, t = V rho */
void orc_se3_exp(const double xi[6], double T[12]) {
  const double* rho = xi;
  const double* phi = xi + 3;
  const double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
  double A, B, C, P[9], P2[9];
  so3_coeffs(th, &A, &B, &C);
  skew3(phi, P);
  m3_mul(P, P, P2);
  double R[9], V[9];
  for (int i = 0; i < 9; ++i) {
    const double I = (i % 4 == 0) ? 1.0 : 0.0;
    R[i] = I + A * P[i] + B * P2[i];
    V[i] = I + B * P[i] + C * P2[i];
  }
  double t[3];
  m3_vec(V, rho, t);
  for (int i = 0; i < 9; ++i) T[i] = R[i];
  for (int i = 0; i < 3; ++i) T[9 + i] = t[i];
}

void orc_se3_log(const double T[12], double xi[6]) {
  const double* R = T;
  double w[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]}; /* vee(R - R^T) */
  const double s = 0.5 * sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  const double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
  const double th = atan2(s, c);
  double phi[3];
  if (th < 1e-6) {
    for (int i = 0; i < 3; ++i) phi[i] = 0.5 * w[i] * (1.0 + th * th / 6.0);
  } else if (th < M_PI - 1e-6) {
    for (int i = 0; i < 3; ++i) phi[i] = th / (2.0 * sin(th)) * w[i];
  } else {
    /* near pi: axis from the largest diagonal entry of (R + I)/2 */
    int k = 0;
    if (R[4] > R[0]) k = 1;
    if (R[8] > R[4 * k]) k = 2;
    double a[3];
    for (int i = 0; i < 3; ++i) a[i] = 0.5 * (R[3 * i + k] + R[3 * k + i]);
    a[k] = sqrt(0.5 * (R[4 * k] + 1.0));
    for (int i = 0; i < 3; ++i)
      if (i != k) a[i] /= 2.0 * a[k];
    const double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    for (int i = 0; i < 3; ++i) phi[i] = th * a[i] / n;
  }
  const double t2 = th * th;
  double D;
  if (th < 1e-4) D = 1.0 / 12.0 + t2 / 720.0;
  else D = (1.0 - th * sin(th) / (2.0 * (1.0 - cos(th)))) / t2;
  double P[9], P2[9], Vi[9];
  skew3(phi, P);
  m3_mul(P, P, P2);
  for (int i = 0; i < 9; ++i) Vi[i] = ((i % 4 == 0) ? 1.0 : 0.0) - 0.5 * P[i] + D * P2[i];
  m3_vec(Vi, T + 9, xi);
  for (int i = 0; i < 3; ++i) xi[3 + i] = phi[i];
}

/* Closed-form left Jacobian of SE(3), xi = (rho, phi):
 * [[Jl(phi), Q(rho,phi)], [0, Jl(phi)]] (Barfoot, State Estimation for
 * Robotics, the SE(3) left Jacobian and its Q block). J is 6x6 row-major. */
void orc_se3_left_jacobian(const double xi[6], double J[36]) {
  const double* rho = xi;
  const double* phi = xi + 3;
  const double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
  double A, B, C;
  so3_coeffs(th, &A, &B, &C);
  double c1, c2, c3;
  if (th < 1e-3) {
    const double t2 = th * th;
    c1 = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
    c2 = 1.0 / 24.0 - t2 / 720.0 + t2 * t2 / 40320.0;
    c3 = 1.0 / 120.0 - t2 / 2520.0;
  } else {
    const double s = sin(th), c = cos(th);
    c1 = (th - s) / (th * th * th);
    c2 = (th * th + 2.0 * c - 2.0) / (2.0 * th * th * th * th);
    c3 = (2.0 * th - 3.0 * s + th * c) / (2.0 * th * th * th * th * th);
  }
  double P[9], Rh[9], P2[9];
  skew3(phi, P);
  skew3(rho, Rh);
  m3_mul(P, P, P2);
  double Jl[9];
  for (int i = 0; i < 9; ++i) Jl[i] = ((i % 4 == 0) ? 1.0 : 0.0) + B * P[i] + C * P2[i];
  double PR[9], RP[9], PRP[9], PPR[9], RPP[9], PRPP[9], PPRP[9];
  m3_mul(P, Rh, PR);
  m3_mul(Rh, P, RP);
  m3_mul(PR, P, PRP);
  m3_mul(P, PR, PPR);
  m3_mul(RP, P, RPP);
  m3_mul(PRP, P, PRPP);
  m3_mul(P, PRP, PPRP);
  double Q[9];
  for (int i = 0; i < 9; ++i)
    Q[i] = 0.5 * Rh[i] + c1 * (PR[i] + RP[i] + PRP[i]) +
           c2 * (PPR[i] + RPP[i] - 3.0 * PRP[i]) + c3 * (PRPP[i] + PPRP[i]);
  memset(J, 0, sizeof(double) * 36);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      J[6 * r + c] = Jl[3 * r + c];
      J[6 * r + 3 + c] = Q[3 * r + c];
      J[6 * (r + 3) + 3 + c] = Jl[3 * r + c];
    }
}

/* Adam (Kingma & Ba) with bias correction at step t (1-based). */
void orc_adam(int64_t n, double* p, const double* g, double* m, double* v,
              double lr, double beta1, double beta2, double eps, int step) {
  const double bc1 = 1.0 - pow(beta1, step);
  const double bc2 = 1.0 - pow(beta2, step);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    const double mh = m[i] / bc1, vh = v[i] / bc2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/*
 * Pose step (Algorithm 1, "Update poses"; Sec. 3.3: Adam on the camera
 * extrinsics).  g_xi = Jl(xi)^T g_tangent; optional Adam step on xi; then
 * Rt_out = Exp(xi) T0 for every camera.
 */
void orc_pose_update(int32_t n_cams, const double* T0, double* xi,
                     const double* g_tangent, double* g_xi, double* m,
                     double* v, int use_adam, double lr, double beta1,
                     double beta2, double eps, int step, double* Rt_out) {
  for (int i = 0; i < n_cams; ++i) {
    double J[36];
    orc_se3_left_jacobian(xi + 6 * i, J);
    double g[6];
    for (int c = 0; c < 6; ++c) {
      double s = 0.0;
      for (int r = 0; r < 6; ++r) s += J[6 * r + c] * g_tangent[6 * i + r];
      g[c] = s;
    }
    if (g_xi)
      for (int c = 0; c < 6; ++c) g_xi[6 * i + c] = g[c];
    if (use_adam) orc_adam(6, xi + 6 * i, g, m + 6 * i, v + 6 * i, lr, beta1, beta2, eps, step);
    double E[12];
    orc_se3_exp(xi + 6 * i, E);
    const double* R0 = T0 + 12 * i;
    double R[9], t[3];
    m3_mul(E, R0, R);
    m3_vec(E, R0 + 9, t);
    for (int a = 0; a < 3; ++a) t[a] += E[9 + a];
    for (int a = 0; a < 9; ++a) Rt_out[12 * i + a] = R[a];
    for (int a = 0; a < 3; ++a) Rt_out[12 * i + 9 + a] = t[a];
  }
}
