/*
 * adp_oracle.c -- FP64 CPU oracle for the AdpSplit hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. It shares no code, header,
 * table or helper with the CUDA path; the two meet only through the seeded
 * inputs of the `scenes` module.
 *
 * Each function follows the step of the method it names, in the paper's order
 * and notation, with no tiling, fusion or reordering beyond what the step's
 * definition states:
 *   - projection (Sec. 3, Eq. 1 and the 3DGS EWA splatting it builds on),
 *   - per-pixel front-to-back compositing, brute force per pixel (Eq. 1),
 *   - the dominant Gaussian map (Eq. 5),
 *   - the min-max normalised L1 error map, mask and bands (Eq. 6, Sec. 4.1),
 *   - erosion, 8-connected error regions and the area filter (Eqs. 7-8),
 *   - region statistics (Sec. 4.1),
 *   - child initialisation (Eqs. 9-10 and Appendix A),
 *   - cross-view child merging and the N_max cap (Eqs. 11-12, Sec. 4.3),
 *   - parent copy, fallback split and reset (Sec. 5.1, Eqs. 3-4),
 *   - the gradient of the L1 training loss (complex-step derivative of the
 *     forward defined here), and one Adam step.
 *
 * Floating point is FP64 throughout, with one exception the method forces:
 * where a float decides an integer (the mask M, the band B), the decision is
 * taken in FP32, the precision of the image the path stores, so that both
 * implementations decide on identical float32 values.
 *
 * Parity status: every function here has a pin in the CPU test suite (closed
 * forms, library special cases, brute force, invariants, finite differences).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Types                                                                      */
/* ------------------------------------------------------------------------ */

/* OpenCV pinhole camera: x right, y down, z forward. R is world->camera,
 * row-major; a world point X maps to camera point R X + t. Pixel (x, y) has
 * its centre at continuous image coordinate (x, y). */
typedef struct orc_camera {
  int32_t width, height;
  double fx, fy, px, py;
  double R[9];
  double t[3];
} orc_camera;

typedef struct orc_config {
  double near_plane; /* cull at camera z <= near_plane */
  double low_pass;   /* added to the diagonal of the 2D covariance */
  double alpha_min;  /* a Gaussian contributes iff o*exp(power) >= alpha_min */
  double alpha_max;  /* alpha is clamped to alpha_max */
  double t_min;      /* stop before blending when T*(1-alpha) < t_min */
  /* Tie bands (absolute). A pixel is a tie when, among the Gaussians it tests,
   * some alpha_raw lies within tie_alpha_min of alpha_min (bit 1) or within
   * tie_alpha_max of alpha_max (bit 4), some stop test T (1 - alpha) lies within
   * tie_stop of t_min (bit 2), or the two largest weights T alpha differ by less
   * than tie_margin (bit 8). Misses with alpha_raw >= alpha_min - tie_capture are
   * kept (not blended) so that their distance to alpha_min is reported. */
  double tie_alpha_min, tie_stop, tie_alpha_max, tie_margin, tie_capture;
  int32_t tile_w, tile_h;
} orc_config;

typedef struct orc_split_config {
  double gamma_d;     /* merge distance threshold (Eq. 11) */
  double gamma_c;     /* merge colour threshold (Eq. 11) */
  double eps_t;       /* epsilon in the denominator of Eq. 10 */
  double eta;         /* vanilla split shrink factor (Eq. 4) */
  double scale_floor; /* lower bound on child scales */
  int32_t n_max;      /* child cap per parent */
  int32_t pad;
} orc_split_config;

enum { ORC_KEEP = 0, ORC_ADAPTIVE = 1, ORC_FALLBACK = 2, ORC_RESET = 3 };

/* Flat per-Gaussian parameter vector theta (length 11 + 3K):
 *   [0..2] mean, [3] opacity logit, [4..6] log-scale, [7..10] quaternion
 *   (w, x, y, z), [11 + 3k + ch] SH coefficient k of channel ch. */
#define TH_MEAN 0
#define TH_LOGIT 3
#define TH_LOGS 4
#define TH_QUAT 7
#define TH_SH 11

/* ------------------------------------------------------------------------ */
/* Spherical harmonics (real basis, 3DGS sign convention)                     */
/* ------------------------------------------------------------------------ */

/* Normalisation constants of the real spherical harmonics up to degree 3,
 * written from their closed forms. The signs follow the 3DGS basis. */
static double shc(int k) {
  const double pi = M_PI;
  switch (k) {
    case 0: return 0.5 * sqrt(1.0 / pi);
    case 1: return -sqrt(3.0 / (4.0 * pi));
    case 2: return sqrt(3.0 / (4.0 * pi));
    case 3: return -sqrt(3.0 / (4.0 * pi));
    case 4: return 0.5 * sqrt(15.0 / pi);
    case 5: return -0.5 * sqrt(15.0 / pi);
    case 6: return 0.25 * sqrt(5.0 / pi);
    case 7: return -0.5 * sqrt(15.0 / pi);
    case 8: return 0.25 * sqrt(15.0 / pi);
    case 9: return -0.25 * sqrt(35.0 / (2.0 * pi));
    case 10: return 0.5 * sqrt(105.0 / pi);
    case 11: return -0.25 * sqrt(21.0 / (2.0 * pi));
    case 12: return 0.25 * sqrt(7.0 / pi);
    case 13: return -0.25 * sqrt(21.0 / (2.0 * pi));
    case 14: return 0.25 * sqrt(105.0 / pi);
    case 15: return -0.25 * sqrt(35.0 / (2.0 * pi));
  }
  return 0.0;
}

/* Basis functions Y_k(d) for a unit direction d = (x, y, z), k < (deg+1)^2. */
static void sh_basis_c(int deg, cplx x, cplx y, cplx z, cplx* Y) {
  Y[0] = shc(0);
  if (deg < 1) return;
  Y[1] = shc(1) * y;
  Y[2] = shc(2) * z;
  Y[3] = shc(3) * x;
  if (deg < 2) return;
  cplx xx = x * x, yy = y * y, zz = z * z;
  Y[4] = shc(4) * x * y;
  Y[5] = shc(5) * y * z;
  Y[6] = shc(6) * (2.0 * zz - xx - yy);
  Y[7] = shc(7) * x * z;
  Y[8] = shc(8) * (xx - yy);
  if (deg < 3) return;
  Y[9] = shc(9) * y * (3.0 * xx - yy);
  Y[10] = shc(10) * x * y * z;
  Y[11] = shc(11) * y * (4.0 * zz - xx - yy);
  Y[12] = shc(12) * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
  Y[13] = shc(13) * x * (4.0 * zz - xx - yy);
  Y[14] = shc(14) * z * (xx - yy);
  Y[15] = shc(15) * x * (xx - 3.0 * yy);
}

ORC_API void orc_sh_basis(int32_t deg, int64_t n, const double* dirs, double* out) {
  int K = (deg + 1) * (deg + 1);
  for (int64_t i = 0; i < n; ++i) {
    cplx Y[16];
    sh_basis_c(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], Y);
    for (int k = 0; k < K; ++k) out[i * K + k] = creal(Y[k]);
  }
}

/* ------------------------------------------------------------------------ */
/* Rotations                                                                  */
/* ------------------------------------------------------------------------ */

/* Rotation matrix (row-major) of the unit quaternion (w, x, y, z). */
static void quat_to_rot_c(cplx w, cplx x, cplx y, cplx z, cplx* R) {
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

static void quat_to_rot(const double* q, double* R) {
  double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  cplx Rc[9];
  quat_to_rot_c(q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq, Rc);
  for (int i = 0; i < 9; ++i) R[i] = creal(Rc[i]);
}

ORC_API void orc_quat_to_rot(int64_t n, const double* q, double* R) {
  for (int64_t i = 0; i < n; ++i) quat_to_rot(q + 4 * i, R + 9 * i);
}

/* Unit quaternion (w, x, y, z) with w >= 0 of a proper rotation (row-major). */
static void rot_to_quat(const double* R, double* q) {
  double tr = R[0] + R[4] + R[8];
  double w, x, y, z;
  if (tr > 0.0) {
    double S = 2.0 * sqrt(tr + 1.0);
    w = 0.25 * S; x = (R[7] - R[5]) / S; y = (R[2] - R[6]) / S; z = (R[3] - R[1]) / S;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    double S = 2.0 * sqrt(1.0 + R[0] - R[4] - R[8]);
    w = (R[7] - R[5]) / S; x = 0.25 * S; y = (R[1] + R[3]) / S; z = (R[2] + R[6]) / S;
  } else if (R[4] > R[8]) {
    double S = 2.0 * sqrt(1.0 + R[4] - R[0] - R[8]);
    w = (R[2] - R[6]) / S; x = (R[1] + R[3]) / S; y = 0.25 * S; z = (R[5] + R[7]) / S;
  } else {
    double S = 2.0 * sqrt(1.0 + R[8] - R[0] - R[4]);
    w = (R[3] - R[1]) / S; x = (R[2] + R[6]) / S; y = (R[5] + R[7]) / S; z = 0.25 * S;
  }
  double nq = sqrt(w * w + x * x + y * y + z * z);
  if (w < 0) nq = -nq;
  q[0] = w / nq; q[1] = x / nq; q[2] = y / nq; q[3] = z / nq;
}

ORC_API void orc_rot_to_quat(int64_t n, const double* R, double* q) {
  for (int64_t i = 0; i < n; ++i) rot_to_quat(R + 9 * i, q + 4 * i);
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* ------------------------------------------------------------------------ */
/* Projection (EWA splatting of one Gaussian into one camera)                 */
/* ------------------------------------------------------------------------ */

/* Projects the Gaussian with parameters th (length 11 + 3K, complex so the
 * gradient can be taken by complex step) into camera cam. Returns 0 if the
 * Gaussian is culled (behind the near plane, degenerate 2D covariance, or an
 * opacity below alpha_min so that no pixel can reach the contribution
 * threshold). out = (mean2d x, mean2d y, conic A, conic B, conic C, opacity,
 * r, g, b); the conic is the inverse 2D covariance [[A, B], [B, C]]. */
static int proj_core(const orc_camera* cam, const orc_config* cfg, int deg, const cplx* th,
                     cplx* out, double* depth, double* cov, int* clamped) {
  const double* Rw = cam->R;
  const double* tw = cam->t;
  int K = (deg + 1) * (deg + 1);
  cplx pc[3];
  for (int r = 0; r < 3; ++r)
    pc[r] = Rw[3 * r] * th[0] + Rw[3 * r + 1] * th[1] + Rw[3 * r + 2] * th[2] + tw[r];
  cplx z = pc[2];
  if (creal(z) <= cfg->near_plane) return 0;

  cplx o = 1.0 / (1.0 + cexp(-th[TH_LOGIT]));
  if (creal(o) < cfg->alpha_min) return 0;

  /* 3D covariance Sigma = R S S^T R^T */
  cplx s[3] = {cexp(th[TH_LOGS]), cexp(th[TH_LOGS + 1]), cexp(th[TH_LOGS + 2])};
  cplx qn = csqrt(th[7] * th[7] + th[8] * th[8] + th[9] * th[9] + th[10] * th[10]);
  cplx Rg[9];
  quat_to_rot_c(th[7] / qn, th[8] / qn, th[9] / qn, th[10] / qn, Rg);
  cplx Sig[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k) acc += Rg[3 * i + k] * s[k] * s[k] * Rg[3 * j + k];
      Sig[3 * i + j] = acc;
    }

  /* Local affine approximation J of the perspective map at the camera-space
   * mean, with x/z and y/z clamped to 1.3x the half field of view. */
  double limx = 1.3 * (double)cam->width / (2.0 * cam->fx);
  double limy = 1.3 * (double)cam->height / (2.0 * cam->fy);
  cplx txz = pc[0] / z, tyz = pc[1] / z;
  if (creal(txz) > limx) txz = limx;
  else if (creal(txz) < -limx) txz = -limx;
  if (creal(tyz) > limy) tyz = limy;
  else if (creal(tyz) < -limy) tyz = -limy;
  cplx J[6] = {cam->fx / z, 0.0, -cam->fx * txz / z, 0.0, cam->fy / z, -cam->fy * tyz / z};

  /* T = J W, Sigma2D = T Sigma T^T + low_pass I */
  cplx T[6];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k) acc += J[3 * r + k] * Rw[3 * k + c];
      T[3 * r + c] = acc;
    }
  cplx C2[4];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      cplx acc = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) acc += T[3 * r + i] * Sig[3 * i + j] * T[3 * c + j];
      C2[2 * r + c] = acc;
    }
  cplx a = C2[0] + cfg->low_pass, b = C2[1], c = C2[3] + cfg->low_pass;
  cplx det = a * c - b * b;
  if (creal(det) <= 0.0) return 0;

  out[0] = cam->fx * pc[0] / z + cam->px;
  out[1] = cam->fy * pc[1] / z + cam->py;
  out[2] = c / det;
  out[3] = -b / det;
  out[4] = a / det;
  out[5] = o;

  /* View-dependent colour: SH evaluated at the unit direction from the camera
   * centre to the mean, plus 0.5, clamped below at 0. */
  double oc[3];
  for (int i = 0; i < 3; ++i) oc[i] = -(Rw[i] * tw[0] + Rw[3 + i] * tw[1] + Rw[6 + i] * tw[2]);
  cplx d[3] = {th[0] - oc[0], th[1] - oc[1], th[2] - oc[2]};
  cplx len = csqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  cplx Y[16];
  sh_basis_c(deg, d[0] / len, d[1] / len, d[2] / len, Y);
  for (int ch = 0; ch < 3; ++ch) {
    cplx v = 0.5;
    for (int k = 0; k < K; ++k) v += th[TH_SH + 3 * k + ch] * Y[k];
    int cl = creal(v) < 0.0;
    if (clamped) clamped[ch] = cl;
    out[6 + ch] = cl ? 0.0 : v;
  }
  if (depth) *depth = creal(z);
  if (cov) { cov[0] = creal(a); cov[1] = creal(b); cov[2] = creal(c); }
  return 1;
}

/* Axis-aligned pixel box of the ellipse o*exp(-0.5 d^T C d) >= alpha_min, i.e.
 * d^T C d <= k with k = 2 ln(o / alpha_min); its half-widths are sqrt(k Sxx)
 * and sqrt(k Syy) of the 2D covariance. Returns 0 if the box misses the
 * image. box = (x0, x1, y0, y1) inclusive. */
static int pixel_box(const orc_camera* cam, const orc_config* cfg, double mx, double my,
                     double opacity, const double* cov, int32_t* box) {
  double k = 2.0 * log(opacity / cfg->alpha_min);
  if (k < 0.0) k = 0.0;
  double hx = sqrt(k * cov[0]), hy = sqrt(k * cov[2]);
  double x0 = ceil(mx - hx), x1 = floor(mx + hx), y0 = ceil(my - hy), y1 = floor(my + hy);
  if (x0 < 0) x0 = 0;
  if (y0 < 0) y0 = 0;
  if (x1 > cam->width - 1) x1 = cam->width - 1;
  if (y1 > cam->height - 1) y1 = cam->height - 1;
  if (x0 > x1 || y0 > y1) return 0;
  box[0] = (int32_t)x0; box[1] = (int32_t)x1; box[2] = (int32_t)y0; box[3] = (int32_t)y1;
  return 1;
}

/* Projects n Gaussians. tiles[i] = number of tiles the pixel box touches
 * (0 = not rendered); rect = tile range (tx0, tx1, ty0, ty1) inclusive. */
ORC_API void orc_project(int64_t n, int32_t deg, const double* theta, const orc_camera* cam,
                         const orc_config* cfg, double* mean2d, double* cov2d, double* conic,
                         double* depth, double* opacity, double* rgb, int32_t* clamped,
                         int32_t* box, int32_t* rect, int32_t* tiles) {
  int P = 11 + 3 * (deg + 1) * (deg + 1);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    cplx th[59];
    for (int p = 0; p < P; ++p) th[p] = theta[i * P + p];
    cplx out[9];
    double dep = 0, cov[3] = {0, 0, 0};
    int cl[3] = {0, 0, 0};
    int vis = proj_core(cam, cfg, deg, th, out, &dep, cov, cl);
    int32_t bx[4] = {0, -1, 0, -1};
    if (vis) vis = pixel_box(cam, cfg, creal(out[0]), creal(out[1]), creal(out[5]), cov, bx);
    mean2d[2 * i] = creal(out[0]) * vis;
    mean2d[2 * i + 1] = creal(out[1]) * vis;
    for (int j = 0; j < 3; ++j) {
      cov2d[3 * i + j] = vis ? cov[j] : 0.0;
      conic[3 * i + j] = vis ? creal(out[2 + j]) : 0.0;
      rgb[3 * i + j] = vis ? creal(out[6 + j]) : 0.0;
      if (clamped) clamped[3 * i + j] = vis ? cl[j] : 0;
    }
    depth[i] = vis ? dep : 0.0;
    opacity[i] = vis ? creal(out[5]) : 0.0;
    for (int j = 0; j < 4; ++j) box[4 * i + j] = bx[j];
    if (vis) {
      rect[4 * i + 0] = bx[0] / cfg->tile_w;
      rect[4 * i + 1] = bx[1] / cfg->tile_w;
      rect[4 * i + 2] = bx[2] / cfg->tile_h;
      rect[4 * i + 3] = bx[3] / cfg->tile_h;
      tiles[i] = (rect[4 * i + 1] - rect[4 * i] + 1) * (rect[4 * i + 3] - rect[4 * i + 2] + 1);
    } else {
      rect[4 * i] = rect[4 * i + 2] = 0;
      rect[4 * i + 1] = rect[4 * i + 3] = -1;
      tiles[i] = 0;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Per-pixel compositing (Eq. 1) and the dominant map (Eq. 5)                */
/* ------------------------------------------------------------------------ */

typedef struct {
  double depth;
  int32_t id;
  int32_t include; /* 1: alpha_raw >= alpha_min; 0: a near-threshold miss kept for its distance */
  double alpha_raw;
} contrib_t;

static int contrib_cmp(const void* a, const void* b) {
  const contrib_t* x = (const contrib_t*)a;
  const contrib_t* y = (const contrib_t*)b;
  if (x->depth < y->depth) return -1;
  if (x->depth > y->depth) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

typedef struct {
  const double *mean2d, *conic, *depth, *opacity, *rgb;
  const int32_t *box, *tiles;
} proj_view_t;

/* alpha_raw of Gaussian i at pixel (x, y): o * exp(-0.5 d^T C d); -1 if the
 * quadratic form is negative (never for a positive-definite conic). */
static double alpha_raw_at(const proj_view_t* pv, int64_t i, int x, int y) {
  double dx = pv->mean2d[2 * i] - x, dy = pv->mean2d[2 * i + 1] - y;
  const double* C = pv->conic + 3 * i;
  double power = -0.5 * (C[0] * dx * dx + C[2] * dy * dy) - C[1] * dx * dy;
  if (power > 0.0) return -1.0;
  return pv->opacity[i] * exp(power);
}

/* Adds Gaussian i to the pixel's list if it contributes, or records a near
 * miss (within tie_capture below alpha_min) so its distance can be reported. */
static void consider(const proj_view_t* pv, const orc_config* cfg, int64_t i, int x, int y,
                     contrib_t* list, int* cnt) {
  if (pv->tiles[i] <= 0) return;
  const int32_t* b = pv->box + 4 * i;
  if (x < b[0] || x > b[1] || y < b[2] || y > b[3]) return;
  double a = alpha_raw_at(pv, i, x, y);
  if (a < 0.0) return;
  int inc = a >= cfg->alpha_min;
  if (!inc && a < cfg->alpha_min - cfg->tie_capture) return;
  contrib_t c = {pv->depth[i], (int32_t)i, inc, a};
  list[(*cnt)++] = c;
}

typedef struct {
  double rgb[3];
  double T;
  int32_t n_contrib;
  int32_t dominant;
  int32_t second;
  double margin;
  double dist[4]; /* distances to alpha_min, t_min, alpha_max; the margin */
  int32_t tie;
} pixel_out_t;

/* Front-to-back compositing of the depth-sorted list (Eq. 1): alpha =
 * min(alpha_max, alpha_raw); stop before blending a Gaussian once
 * T (1 - alpha) < t_min. The dominant Gaussian maximises T alpha (Eq. 5); a
 * strict comparison keeps the earliest on ties. The distances cover every
 * Gaussian tested up to and including the one that stops the pixel. Tie bits: 1
 * alpha threshold, 2 stop threshold, 4 alpha clamp, 8 dominant margin. */
static void composite(const proj_view_t* pv, const orc_config* cfg, const double* bg,
                      const contrib_t* list, int cnt, pixel_out_t* po) {
  double T = 1.0, col[3] = {0, 0, 0}, best = -1.0, second = -1.0;
  int dom = -1, sec = -1, n = 0, tie = 0;
  double d_amin = 1e300, d_stop = 1e300, d_amax = 1e300;
  for (int k = 0; k < cnt; ++k) {
    double a_raw = list[k].alpha_raw;
    d_amin = fmin(d_amin, fabs(a_raw - cfg->alpha_min));
    if (!list[k].include) continue;
    d_amax = fmin(d_amax, fabs(a_raw - cfg->alpha_max));
    double a = a_raw < cfg->alpha_max ? a_raw : cfg->alpha_max;
    double test = T * (1.0 - a);
    d_stop = fmin(d_stop, fabs(test - cfg->t_min));
    if (test < cfg->t_min) break;
    double w = T * a;
    const double* c = pv->rgb + 3 * (int64_t)list[k].id;
    for (int ch = 0; ch < 3; ++ch) col[ch] += w * c[ch];
    if (w > best) {
      second = best; sec = dom; best = w; dom = list[k].id;
    } else if (w > second) {
      second = w; sec = list[k].id;
    }
    T = test;
    ++n;
  }
  for (int ch = 0; ch < 3; ++ch) po->rgb[ch] = col[ch] + T * bg[ch];
  po->T = T;
  po->n_contrib = n;
  po->dominant = dom;
  po->second = sec;
  po->margin = (dom >= 0 && sec >= 0) ? best - second : 1e300;
  if (d_amin < cfg->tie_alpha_min) tie |= 1;
  if (d_stop < cfg->tie_stop) tie |= 2;
  if (d_amax < cfg->tie_alpha_max) tie |= 4;
  if (po->margin < cfg->tie_margin) tie |= 8;
  po->dist[0] = d_amin;
  po->dist[1] = d_stop;
  po->dist[2] = d_amax;
  po->dist[3] = po->margin;
  po->tie = tie;
}

static void store_pixel(const pixel_out_t* po, int64_t j, double* out_rgb, double* out_T,
                        int32_t* out_n, int32_t* out_dom, int32_t* out_second,
                        double* out_dist, int32_t* out_tie) {
  for (int ch = 0; ch < 3; ++ch) out_rgb[3 * j + ch] = po->rgb[ch];
  out_T[j] = po->T;
  out_n[j] = po->n_contrib;
  out_dom[j] = po->dominant;
  if (out_second) out_second[j] = po->second;
  if (out_dist)
    for (int e = 0; e < 4; ++e) out_dist[4 * j + e] = po->dist[e];
  if (out_tie) out_tie[j] = po->tie;
}

/* Renders pixels of one view. If pix is NULL every pixel is rendered in
 * row-major order, gathering each pixel's candidates from a coarse grid of
 * cells indexed by the Gaussians' own pixel boxes (a pruning of the candidate
 * scan only: each pixel is still composited from exactly the Gaussians whose
 * alpha reaches the threshold there). Otherwise the n_pix linear pixel indices
 * in pix are rendered by brute force, testing every Gaussian. */
ORC_API void orc_render(int64_t n, const double* mean2d, const double* conic, const double* depth,
                        const double* opacity, const double* rgb, const int32_t* box,
                        const int32_t* tiles, int32_t W, int32_t H, const double* bg,
                        const orc_config* cfg, int64_t n_pix, const int64_t* pix,
                        double* out_rgb, double* out_T, int32_t* out_n, int32_t* out_dom,
                        int32_t* out_second, double* out_dist, int32_t* out_tie) {
  proj_view_t pv = {mean2d, conic, depth, opacity, rgb, box, tiles};
  if (pix) {
#pragma omp parallel
    {
      contrib_t* list = (contrib_t*)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
      for (int64_t j = 0; j < n_pix; ++j) {
        int x = (int)(pix[j] % W), y = (int)(pix[j] / W);
        int cnt = 0;
        for (int64_t i = 0; i < n; ++i) consider(&pv, cfg, i, x, y, list, &cnt);
        qsort(list, (size_t)cnt, sizeof(contrib_t), contrib_cmp);
        pixel_out_t po;
        composite(&pv, cfg, bg, list, cnt, &po);
        store_pixel(&po, j, out_rgb, out_T, out_n, out_dom, out_second, out_dist, out_tie);
      }
      free(list);
    }
    return;
  }
  /* Candidate lists per 16x16 cell of pixels, from the Gaussians' boxes. */
  const int CS = 16;
  int cw = (W + CS - 1) / CS, ch_ = (H + CS - 1) / CS;
  int64_t ncell = (int64_t)cw * ch_;
  int64_t* start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    if (tiles[i] <= 0) continue;
    const int32_t* b = box + 4 * i;
    for (int cy = b[2] / CS; cy <= b[3] / CS; ++cy)
      for (int cx = b[0] / CS; cx <= b[1] / CS; ++cx) start[(int64_t)cy * cw + cx + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
  int32_t* ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)(start[ncell] > 0 ? start[ncell] : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
  memcpy(fill, start, sizeof(int64_t) * (size_t)ncell);
  for (int64_t i = 0; i < n; ++i) {
    if (tiles[i] <= 0) continue;
    const int32_t* b = box + 4 * i;
    for (int cy = b[2] / CS; cy <= b[3] / CS; ++cy)
      for (int cx = b[0] / CS; cx <= b[1] / CS; ++cx) ids[fill[(int64_t)cy * cw + cx]++] = (int32_t)i;
  }
  int64_t maxlen = 1;
  for (int64_t c = 0; c < ncell; ++c)
    if (start[c + 1] - start[c] > maxlen) maxlen = start[c + 1] - start[c];
#pragma omp parallel
  {
    contrib_t* list = (contrib_t*)malloc(sizeof(contrib_t) * (size_t)maxlen);
#pragma omp for schedule(dynamic, 64)
    for (int64_t j = 0; j < (int64_t)W * H; ++j) {
      int x = (int)(j % W), y = (int)(j / W);
      int64_t c = (int64_t)(y / CS) * cw + x / CS;
      int cnt = 0;
      for (int64_t e = start[c]; e < start[c + 1]; ++e) consider(&pv, cfg, ids[e], x, y, list, &cnt);
      qsort(list, (size_t)cnt, sizeof(contrib_t), contrib_cmp);
      pixel_out_t po;
      composite(&pv, cfg, bg, list, cnt, &po);
      store_pixel(&po, j, out_rgb, out_T, out_n, out_dom, out_second, out_dist, out_tie);
    }
    free(list);
  }
  free(start);
  free(ids);
  free(fill);
}

/* Per-tile instance lists by definition: for every tile (row-major), the
 * Gaussians whose tile rectangle covers it, ordered by (depth, id). Returns
 * the number of instances; writes tile_start[n_tiles + 1] and inst[] (if
 * capacity allows). Keys are float32 depths, as the CUDA path sorts them. */
typedef struct { float depth; int32_t id; } depth_key_t;
static int depth_key_cmp(const void* a, const void* b) {
  const depth_key_t* x = (const depth_key_t*)a;
  const depth_key_t* y = (const depth_key_t*)b;
  if (x->depth < y->depth) return -1;
  if (x->depth > y->depth) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

ORC_API int64_t orc_tile_lists(int64_t n, const float* depth, const int32_t* rect,
                               const int32_t* tiles, int32_t tiles_x, int32_t tiles_y,
                               int64_t* tile_start, int64_t cap, int32_t* inst) {
  int64_t nt = (int64_t)tiles_x * tiles_y;
  for (int64_t t = 0; t <= nt; ++t) tile_start[t] = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (tiles[i] <= 0) continue;
    const int32_t* r = rect + 4 * i;
    for (int ty = r[2]; ty <= r[3]; ++ty)
      for (int tx = r[0]; tx <= r[1]; ++tx) tile_start[(int64_t)ty * tiles_x + tx + 1]++;
  }
  for (int64_t t = 0; t < nt; ++t) tile_start[t + 1] += tile_start[t];
  int64_t total = tile_start[nt];
  if (total > cap || !inst) return total;
  depth_key_t* keys = (depth_key_t*)malloc(sizeof(depth_key_t) * (size_t)(n > 0 ? n : 1));
  int64_t nv = 0;
  for (int64_t i = 0; i < n; ++i)
    if (tiles[i] > 0) { keys[nv].depth = depth[i]; keys[nv].id = (int32_t)i; ++nv; }
  qsort(keys, (size_t)nv, sizeof(depth_key_t), depth_key_cmp);
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt > 0 ? nt : 1));
  memcpy(fill, tile_start, sizeof(int64_t) * (size_t)nt);
  for (int64_t k = 0; k < nv; ++k) {
    const int32_t* r = rect + 4 * keys[k].id;
    for (int ty = r[2]; ty <= r[3]; ++ty)
      for (int tx = r[0]; tx <= r[1]; ++tx) inst[fill[(int64_t)ty * tiles_x + tx]++] = keys[k].id;
  }
  free(keys);
  free(fill);
  return total;
}

/* ------------------------------------------------------------------------ */
/* Error map, mask, bands (Eq. 6, Sec. 4.1), erosion, per-Gaussian stats     */
/* ------------------------------------------------------------------------ */

/* raw(u) = |I^ - I_gt|_1 summed over the three channels; E = (raw - min) /
 * (max - min) over the view (E = 0 if max == min); M = [E > tau]; band
 * B = min(L - 1, floor(L (E - tau) / (1 - tau))) for M = 1, else 0. All in
 * float32 arithmetic (see the header). */
ORC_API void orc_error_map(int32_t W, int32_t H, const float* img, const float* tgt, float tau,
                           int32_t L, float* out_raw, float* out_E, uint8_t* out_M,
                           uint8_t* out_B, float* out_minmax) {
  int64_t P = (int64_t)W * H;
  float mn = INFINITY, mx = -INFINITY;
  for (int64_t u = 0; u < P; ++u) {
    float d0 = fabsf(img[3 * u] - tgt[3 * u]);
    float d1 = fabsf(img[3 * u + 1] - tgt[3 * u + 1]);
    float d2 = fabsf(img[3 * u + 2] - tgt[3 * u + 2]);
    float r = (d0 + d1) + d2;
    out_raw[u] = r;
    if (r < mn) mn = r;
    if (r > mx) mx = r;
  }
  if (P == 0) { mn = 0.0f; mx = 0.0f; }
  out_minmax[0] = mn;
  out_minmax[1] = mx;
  float range = mx - mn;
  float one_minus_tau = 1.0f - tau;
  for (int64_t u = 0; u < P; ++u) {
    float e = range > 0.0f ? (out_raw[u] - mn) / range : 0.0f;
    out_E[u] = e;
    uint8_t m = e > tau;
    out_M[u] = m;
    uint8_t b = 0;
    if (m) {
      float t = ((e - tau) * (float)L) / one_minus_tau;
      int bi = (int)floorf(t);
      if (bi > L - 1) bi = L - 1;
      if (bi < 0) bi = 0;
      b = (uint8_t)bi;
    }
    out_B[u] = b;
  }
}

/* Erosion of the mask by a (2r+1) x (2r+1) square; pixels outside the image
 * count as set, so the image border does not erode. r = 0 is the identity. */
ORC_API void orc_erode(int32_t W, int32_t H, const uint8_t* M, int32_t r, uint8_t* out) {
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      uint8_t v = M[(int64_t)y * W + x];
      for (int dy = -r; dy <= r && v; ++dy)
        for (int dx = -r; dx <= r && v; ++dx) {
          int xx = x + dx, yy = y + dy;
          if (xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
          if (!M[(int64_t)yy * W + xx]) v = 0;
        }
      out[(int64_t)y * W + x] = v;
    }
}

/* Error pixels attributed to each Gaussian (accumulates into count/mass):
 * pixels with M = 1 (before erosion) whose dominant Gaussian is i. */
ORC_API void orc_gauss_stats(int64_t P, const uint8_t* M, const int32_t* D, const float* E,
                             int64_t n, int32_t* count, double* mass) {
  for (int64_t u = 0; u < P; ++u) {
    if (!M[u] || D[u] < 0 || D[u] >= n) continue;
    count[D[u]] += 1;
    mass[D[u]] += (double)E[u];
  }
}

typedef struct { double mass; int32_t id; } mass_key_t;
static int mass_key_cmp(const void* a, const void* b) {
  const mass_key_t* x = (const mass_key_t*)a;
  const mass_key_t* y = (const mass_key_t*)b;
  if (x->mass > y->mass) return -1;
  if (x->mass < y->mass) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

/* The k Gaussians with the largest error mass, ties to the lower id, returned
 * in ascending id order. */
ORC_API void orc_topk_mass(int64_t n, const double* mass, int64_t k, int32_t* out_ids) {
  mass_key_t* keys = (mass_key_t*)malloc(sizeof(mass_key_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) { keys[i].mass = mass[i]; keys[i].id = (int32_t)i; }
  qsort(keys, (size_t)n, sizeof(mass_key_t), mass_key_cmp);
  uint8_t* pick = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int64_t j = 0; j < k && j < n; ++j) pick[keys[j].id] = 1;
  int64_t o = 0;
  for (int64_t i = 0; i < n; ++i)
    if (pick[i]) out_ids[o++] = (int32_t)i;
  free(keys);
  free(pick);
}

/* ------------------------------------------------------------------------ */
/* Error regions (Eqs. 7-8) and region statistics                             */
/* ------------------------------------------------------------------------ */

static int32_t uf_find(int32_t* par, int32_t a) {
  while (par[a] != a) a = par[a];
  return a;
}

/* Union that always hangs the larger root under the smaller one, so each
 * component's final root is its smallest linear pixel index. */
static void uf_union(int32_t* par, int32_t a, int32_t b) {
  a = uf_find(par, a);
  b = uf_find(par, b);
  if (a < b) par[b] = a;
  else if (b < a) par[a] = b;
}

/* Covariance entry (A Sab - Sa Sb) / A^2 from exact integer sums. */
static double exact_cov(int64_t A, int64_t Sab, int64_t Sa, int64_t Sb) {
  __int128 num = (__int128)A * Sab - (__int128)Sa * Sb;
  return (double)num / ((double)A * (double)A);
}

/* Regions of one view. A pixel takes part iff its eroded mask is set and its
 * dominant Gaussian is a split candidate; two such pixels are joined when they
 * are 8-neighbours with the same dominant Gaussian and the same band. Each
 * region is labelled by its smallest linear pixel index y*W + x. Regions with
 * area >= m_min are kept, in ascending label order, with their statistics:
 *   stats = (cx, cy, cov_xx, cov_xy, cov_yy, e1x, e1y, sigma1, sigma2, r, g, b)
 * centroid, population covariance, the major PCA axis e1 (sign chosen with
 * e1x > 0, or e1y > 0 when e1x = 0), standard deviations along e1 and
 * e2 = (-e1y, e1x), and the target RGB at the pixel nearest the centroid.
 * labels[u] receives the label of every participating pixel (before the area
 * filter), -1 elsewhere. Returns the number of kept regions; only the first
 * cap are written. */
ORC_API int64_t orc_regions(int32_t view, int32_t W, int32_t H, const uint8_t* Mero,
                            const uint8_t* B, const int32_t* D, int64_t n,
                            const uint8_t* cand_flag, const float* tgt, int32_t m_min,
                            int32_t* labels, int64_t cap, int32_t* r_view, int32_t* r_parent,
                            int32_t* r_label, int32_t* r_band, int64_t* r_mom,
                            double* r_stats) {
  int64_t P = (int64_t)W * H;
  int32_t* par = labels;
  for (int64_t u = 0; u < P; ++u) {
    int ok = Mero[u] && D[u] >= 0 && D[u] < n && cand_flag[D[u]];
    par[u] = ok ? (int32_t)u : -1;
  }
  const int nb[4][2] = {{-1, 0}, {-1, -1}, {0, -1}, {1, -1}};
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      int64_t u = (int64_t)y * W + x;
      if (par[u] < 0) continue;
      for (int k = 0; k < 4; ++k) {
        int xx = x + nb[k][0], yy = y + nb[k][1];
        if (xx < 0 || yy < 0 || xx >= W) continue;
        int64_t v = (int64_t)yy * W + xx;
        if (par[v] < 0 || D[v] != D[u] || B[v] != B[u]) continue;
        uf_union(par, (int32_t)u, (int32_t)v);
      }
    }
  for (int64_t u = 0; u < P; ++u)
    if (par[u] >= 0) par[u] = uf_find(par, (int32_t)u);

  /* Exact integer moments per label. */
  int64_t nroot = 0;
  int32_t* slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P > 0 ? P : 1));
  for (int64_t u = 0; u < P; ++u)
    if (par[u] == u) slot[u] = (int32_t)nroot++;
  int64_t* mom = (int64_t*)calloc((size_t)(nroot > 0 ? nroot : 1) * 6, sizeof(int64_t));
  for (int64_t u = 0; u < P; ++u) {
    if (par[u] < 0) continue;
    int64_t x = u % W, y = u / W;
    int64_t* m = mom + 6 * (int64_t)slot[par[u]];
    m[0] += 1; m[1] += x; m[2] += y; m[3] += x * x; m[4] += x * y; m[5] += y * y;
  }
  int64_t kept = 0;
  for (int64_t u = 0; u < P; ++u) {
    if (par[u] != u) continue;
    const int64_t* m = mom + 6 * (int64_t)slot[u];
    if (m[0] < m_min) continue;
    if (kept < cap) {
      int64_t A = m[0];
      double cx = (double)m[1] / (double)A, cy = (double)m[2] / (double)A;
      double cxx = exact_cov(A, m[3], m[1], m[1]);
      double cxy = exact_cov(A, m[4], m[1], m[2]);
      double cyy = exact_cov(A, m[5], m[2], m[2]);
      double th = 0.5 * atan2(2.0 * cxy, cxx - cyy);
      double ex = cos(th), ey = sin(th);
      if (ex < 0.0 || (ex == 0.0 && ey < 0.0)) { ex = -ex; ey = -ey; }
      double l1 = cxx * ex * ex + 2.0 * cxy * ex * ey + cyy * ey * ey;
      double l2 = cxx * ey * ey - 2.0 * cxy * ex * ey + cyy * ex * ex;
      int xi = (int)floor(cx + 0.5), yi = (int)floor(cy + 0.5);
      if (xi < 0) xi = 0;
      if (yi < 0) yi = 0;
      if (xi > W - 1) xi = W - 1;
      if (yi > H - 1) yi = H - 1;
      const float* rgb = tgt + 3 * ((int64_t)yi * W + xi);
      double* s = r_stats + 12 * kept;
      s[0] = cx; s[1] = cy; s[2] = cxx; s[3] = cxy; s[4] = cyy; s[5] = ex; s[6] = ey;
      s[7] = sqrt(l1 > 0 ? l1 : 0); s[8] = sqrt(l2 > 0 ? l2 : 0);
      s[9] = rgb[0]; s[10] = rgb[1]; s[11] = rgb[2];
      r_view[kept] = view;
      r_parent[kept] = D[u];
      r_label[kept] = (int32_t)u;
      r_band[kept] = B[u];
      for (int j = 0; j < 6; ++j) r_mom[6 * kept + j] = m[j];
    }
    ++kept;
  }
  free(slot);
  free(mom);
  return kept;
}

/* ------------------------------------------------------------------------ */
/* Child initialisation (Eqs. 9-10, Appendix A)                               */
/* ------------------------------------------------------------------------ */

static double clip_sym(double x, double a) {
  double m = fabs(x) < a ? fabs(x) : a;
  return x < 0 ? -m : m;
}

static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

/* One child proposal from one retained region of a parent. th: the parent's
 * parameter vector; st: the region's 12 statistics. Outputs the child centre
 * mu, the rotation R = [u1 | u2 | z_v] (row-major, columns are the axes), the
 * scales s, colour rgb and the ray parameter t*. */
ORC_API void orc_child_proposal(const double* th, const orc_camera* cam, const double* st,
                                double eps_t, double scale_floor, double* mu, double* R,
                                double* s, double* rgb, double* tstar) {
  const double* Rw = cam->R;
  const double* tw = cam->t;
  /* Parent: Sigma^-1 = R_p diag(s_p^-2) R_p^T */
  double sp[3] = {exp(th[TH_LOGS]), exp(th[TH_LOGS + 1]), exp(th[TH_LOGS + 2])};
  double Rp[9];
  quat_to_rot(th + TH_QUAT, Rp);
  double A[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += Rp[3 * i + k] * Rp[3 * j + k] / (sp[k] * sp[k]);
      A[3 * i + j] = acc;
    }
  /* Camera centre o_v = -R^T t, camera axes in world coordinates (rows of R). */
  double o[3], u[3], w[3], zv[3];
  for (int i = 0; i < 3; ++i) {
    o[i] = -(Rw[i] * tw[0] + Rw[3 + i] * tw[1] + Rw[6 + i] * tw[2]);
    u[i] = Rw[i];
    w[i] = Rw[3 + i];
    zv[i] = Rw[6 + i];
  }
  /* Ray through the centroid. */
  double dcam[3] = {(st[0] - cam->px) / cam->fx, (st[1] - cam->py) / cam->fy, 1.0};
  double d[3];
  for (int i = 0; i < 3; ++i) d[i] = Rw[i] * dcam[0] + Rw[3 + i] * dcam[1] + Rw[6 + i] * dcam[2];
  double dn = norm3(d);
  for (int i = 0; i < 3; ++i) d[i] /= dn;
  /* t* = b^T A d / (d^T A d + eps), b = mu_i - o_v (Eq. 10) */
  double b[3] = {th[0] - o[0], th[1] - o[1], th[2] - o[2]};
  double Ad[3];
  for (int i = 0; i < 3; ++i) Ad[i] = A[3 * i] * d[0] + A[3 * i + 1] * d[1] + A[3 * i + 2] * d[2];
  double ts = dot3(b, Ad) / (dot3(d, Ad) + eps_t);
  *tstar = ts;
  for (int i = 0; i < 3; ++i) mu[i] = o[i] + ts * d[i];
  /* Image-space PCA axes to world-space axes (Appendix A). */
  double tz = ts / norm3(dcam);
  double smax = sp[0] > sp[1] ? (sp[0] > sp[2] ? sp[0] : sp[2]) : (sp[1] > sp[2] ? sp[1] : sp[2]);
  double e1x = st[5], e1y = st[6], e2x = -st[6], e2y = st[5], s1 = st[7], s2 = st[8];
  double w1x = clip_sym(e1x * s1 * tz / cam->fx, smax * fabs(e1x));
  double w1y = clip_sym(e1y * s1 * tz / cam->fy, smax * fabs(e1y));
  double w2x = clip_sym(e2x * s2 * tz / cam->fx, smax * fabs(e2x));
  double w2y = clip_sym(e2y * s2 * tz / cam->fy, smax * fabs(e2y));
  double a1[3], a2[3];
  for (int i = 0; i < 3; ++i) {
    a1[i] = w1x * u[i] + w1y * w[i];
    a2[i] = w2x * u[i] + w2y * w[i];
  }
  double n1 = norm3(a1), n2 = norm3(a2);
  s[0] = n1 > scale_floor ? n1 : scale_floor;
  s[1] = n2 > scale_floor ? n2 : scale_floor;
  s[2] = s[1];
  /* Gram-Schmidt in the image plane. */
  double u1[3], u2[3];
  if (n1 < 1e-12) {
    for (int i = 0; i < 3; ++i) u1[i] = u[i];
  } else {
    for (int i = 0; i < 3; ++i) u1[i] = a1[i] / n1;
  }
  double proj = dot3(a2, u1), r2[3];
  for (int i = 0; i < 3; ++i) r2[i] = a2[i] - proj * u1[i];
  double nr = norm3(r2);
  if (nr < 1e-12) {
    cross3(zv, u1, u2);
  } else {
    for (int i = 0; i < 3; ++i) u2[i] = r2[i] / nr;
  }
  double c12[3];
  cross3(u1, u2, c12);
  if (dot3(c12, zv) < 0.0)
    for (int i = 0; i < 3; ++i) u2[i] = -u2[i];
  for (int i = 0; i < 3; ++i) {
    R[3 * i + 0] = u1[i];
    R[3 * i + 1] = u2[i];
    R[3 * i + 2] = zv[i];
  }
  for (int i = 0; i < 3; ++i) rgb[i] = st[9 + i];
}

/* ------------------------------------------------------------------------ */
/* Cross-view merging (Eqs. 11-12)                                            */
/* ------------------------------------------------------------------------ */

/* Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations.
 * E is row-major with the eigenvectors as columns. */
static void jacobi3(const double* Ain, double* evals, double* E) {
  double A[9];
  memcpy(A, Ain, sizeof(A));
  for (int i = 0; i < 9; ++i) E[i] = (i % 4 == 0) ? 1.0 : 0.0;
  const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    double dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (off <= 1e-32 * dia || off == 0.0) break;
    for (int pi = 0; pi < 3; ++pi) {
      int p = pairs[pi][0], q = pairs[pi][1];
      double apq = A[3 * p + q];
      if (apq == 0.0) continue;
      double theta = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
      double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      double Jm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
      Jm[3 * p + p] = c; Jm[3 * q + q] = c; Jm[3 * p + q] = s; Jm[3 * q + p] = -s;
      double tmp[9], An[9], En[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double acc = 0;
          for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * Jm[3 * k + j];
          tmp[3 * i + j] = acc;
        }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double acc = 0, acc2 = 0;
          for (int k = 0; k < 3; ++k) {
            acc += Jm[3 * k + i] * tmp[3 * k + j];
            acc2 += E[3 * i + k] * Jm[3 * k + j];
          }
          An[3 * i + j] = acc;
          En[3 * i + j] = acc2;
        }
      memcpy(A, An, sizeof(A));
      memcpy(E, En, sizeof(En));
    }
  }
  evals[0] = A[0]; evals[1] = A[4]; evals[2] = A[8];
}

/* Sigma = R diag(s^2) R^T and Sigma^-1 = R diag(s^-2) R^T (R row-major). */
static void cov_from_rs(const double* R, const double* s, double* Sig, double* Sinv) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0, b = 0;
      for (int k = 0; k < 3; ++k) {
        a += R[3 * i + k] * s[k] * s[k] * R[3 * j + k];
        b += R[3 * i + k] * R[3 * j + k] / (s[k] * s[k]);
      }
      if (Sig) Sig[3 * i + j] = a;
      if (Sinv) Sinv[3 * i + j] = b;
    }
}

static double mahal(const double* Sinv, const double* d) {
  double acc = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) acc += d[i] * Sinv[3 * i + j] * d[j];
  return sqrt(acc > 0 ? acc : 0);
}

/* Merges M proposals of one parent. Two proposals are joined when the
 * symmetric Mahalanobis distance of their centres is <= gamma_d and their
 * colours differ by <= gamma_c in every channel (Eq. 11); groups are the
 * connected components (transitive). Each group's centre and colour are the
 * member means; its covariance has the eigenvectors E of the mean member
 * covariance and, along each e_r, the variance max_m (|e_r^T (mu_m - mu_M)| +
 * sigma_{m,r})^2 with sigma_{m,r} = sqrt(e_r^T Sigma_m e_r) (Eq. 12).
 * Groups are numbered by their first member. Outputs per group: mu, rgb,
 * R (= E with det +1, row-major), s (= sqrt of the variances, floored),
 * Sigma. Returns the number of groups; group_of[m] gives each member's group. */
ORC_API int32_t orc_merge(int32_t M, const double* mu, const double* R, const double* s,
                          const double* rgb, double gamma_d, double gamma_c, double scale_floor,
                          int32_t* group_of, double* g_mu, double* g_rgb, double* g_R,
                          double* g_s, double* g_Sig) {
  double* Sig = (double*)malloc(sizeof(double) * 9 * (size_t)(M > 0 ? M : 1));
  double* Sinv = (double*)malloc(sizeof(double) * 9 * (size_t)(M > 0 ? M : 1));
  int32_t* par = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
  for (int m = 0; m < M; ++m) {
    cov_from_rs(R + 9 * m, s + 3 * m, Sig + 9 * m, Sinv + 9 * m);
    par[m] = m;
  }
  for (int a = 0; a < M; ++a)
    for (int b = a + 1; b < M; ++b) {
      double d[3] = {mu[3 * b] - mu[3 * a], mu[3 * b + 1] - mu[3 * a + 1], mu[3 * b + 2] - mu[3 * a + 2]};
      double dist = mahal(Sinv + 9 * a, d) + mahal(Sinv + 9 * b, d);
      double dc = 0;
      for (int ch = 0; ch < 3; ++ch) {
        double x = fabs(rgb[3 * a + ch] - rgb[3 * b + ch]);
        if (x > dc) dc = x;
      }
      if (dist <= gamma_d && dc <= gamma_c) uf_union(par, a, b);
    }
  int32_t ng = 0;
  int32_t* gid = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
  for (int m = 0; m < M; ++m) {
    int r = uf_find(par, m);
    if (r == m) gid[m] = ng++;
  }
  for (int m = 0; m < M; ++m) group_of[m] = gid[uf_find(par, m)];
  for (int g = 0; g < ng; ++g) {
    int cnt = 0;
    double gm[3] = {0, 0, 0}, gc[3] = {0, 0, 0}, Sb[9] = {0};
    for (int m = 0; m < M; ++m) {
      if (group_of[m] != g) continue;
      ++cnt;
      for (int i = 0; i < 3; ++i) { gm[i] += mu[3 * m + i]; gc[i] += rgb[3 * m + i]; }
      for (int i = 0; i < 9; ++i) Sb[i] += Sig[9 * m + i];
    }
    for (int i = 0; i < 3; ++i) { gm[i] /= cnt; gc[i] /= cnt; }
    for (int i = 0; i < 9; ++i) Sb[i] /= cnt;
    double ev[3], E[9];
    jacobi3(Sb, ev, E);
    double lam[3] = {0, 0, 0};
    for (int m = 0; m < M; ++m) {
      if (group_of[m] != g) continue;
      for (int r = 0; r < 3; ++r) {
        double er[3] = {E[r], E[3 + r], E[6 + r]};
        double dm[3] = {mu[3 * m] - gm[0], mu[3 * m + 1] - gm[1], mu[3 * m + 2] - gm[2]};
        double Se[3];
        for (int i = 0; i < 3; ++i)
          Se[i] = Sig[9 * m + 3 * i] * er[0] + Sig[9 * m + 3 * i + 1] * er[1] + Sig[9 * m + 3 * i + 2] * er[2];
        double sig = sqrt(fmax(dot3(er, Se), 0.0));
        double reach = fabs(dot3(er, dm)) + sig;
        if (reach * reach > lam[r]) lam[r] = reach * reach;
      }
    }
    /* det(E) = +1 */
    double c0[3] = {E[0], E[3], E[6]}, c1[3] = {E[1], E[4], E[7]}, c2[3] = {E[2], E[5], E[8]}, cc[3];
    cross3(c0, c1, cc);
    if (dot3(cc, c2) < 0) { E[2] = -E[2]; E[5] = -E[5]; E[8] = -E[8]; }
    double gs[3];
    for (int r = 0; r < 3; ++r) {
      gs[r] = sqrt(lam[r]);
      if (gs[r] < scale_floor) gs[r] = scale_floor;
    }
    for (int i = 0; i < 3; ++i) { g_mu[3 * g + i] = gm[i]; g_rgb[3 * g + i] = gc[i]; g_s[3 * g + i] = gs[i]; }
    for (int i = 0; i < 9; ++i) g_R[9 * g + i] = E[i];
    if (g_Sig) cov_from_rs(E, gs, g_Sig + 9 * g, NULL);
  }
  free(Sig);
  free(Sinv);
  free(par);
  free(gid);
  return ng;
}

/* ------------------------------------------------------------------------ */
/* The AdpSplit operator: statuses, child counts and the new population       */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t parent, view, label; int64_t idx; } reg_key_t;
static int reg_key_cmp(const void* a, const void* b) {
  const reg_key_t* x = (const reg_key_t*)a;
  const reg_key_t* y = (const reg_key_t*)b;
  if (x->parent != y->parent) return x->parent < y->parent ? -1 : 1;
  if (x->view != y->view) return x->view < y->view ? -1 : 1;
  if (x->label != y->label) return x->label < y->label ? -1 : 1;
  return 0;
}

typedef struct { double extent; int32_t g; } ext_key_t;
static int ext_key_cmp(const void* a, const void* b) {
  const ext_key_t* x = (const ext_key_t*)a;
  const ext_key_t* y = (const ext_key_t*)b;
  if (x->extent > y->extent) return -1;
  if (x->extent < y->extent) return 1;
  return (x->g > y->g) - (x->g < y->g);
}

static double logit_of(double o) { return log(o / (1.0 - o)); }

static void write_child(double* out, int P, int K, const double* mu, const double* R,
                        const double* s, const double* rgb, double parent_logit) {
  memset(out, 0, sizeof(double) * (size_t)P);
  for (int i = 0; i < 3; ++i) out[TH_MEAN + i] = mu[i];
  out[TH_LOGIT] = parent_logit;
  for (int i = 0; i < 3; ++i) out[TH_LOGS + i] = log(s[i]);
  rot_to_quat(R, out + TH_QUAT);
  const double C0 = shc(0);
  for (int ch = 0; ch < 3; ++ch) out[TH_SH + ch] = (rgb[ch] - 0.5) / C0;
  (void)K;
}

/* AdpSplit on the candidate list cand (strictly ascending ids).
 *   count[i]: error pixels attributed to Gaussian i over all sampled views.
 *   regions: kept error regions of all views (view, parent, label, stats).
 *   noise[c][2][3]: standard normal draws for candidate c's fallback children.
 * Status per candidate: FALLBACK (vanilla split into 2) when no view attributes
 * an error pixel to it; RESET (kept unchanged) when pixels are attributed but
 * no region survives; otherwise ADAPTIVE with N_i children: one proposal per
 * region (Eqs. 9-10), merged across views (Eqs. 11-12), capped at the n_max
 * largest by sqrt(det Sigma) (ties to the earlier group), emitted in
 * first-member order, plus a parent copy with opacity o/(N_i + 1).
 * The new population is: every non-candidate and RESET Gaussian in id order
 * (keeping its Adam state), then per candidate in ascending id either
 * [parent copy, children...] (ADAPTIVE) or [child 0, child 1] (FALLBACK),
 * each with zero Adam state. Returns the new size; outputs are written only if
 * the new size fits cap_out. */
ORC_API int64_t orc_split(int64_t n, int32_t deg, const double* theta, const double* adam_m,
                          const double* adam_v, const orc_camera* cams, int32_t n_views,
                          int64_t n_reg, const int32_t* r_view, const int32_t* r_parent,
                          const int32_t* r_label, const double* r_stats, int64_t n_cand,
                          const int32_t* cand, const int32_t* count, const double* noise,
                          const orc_split_config* sc, uint8_t* status, int32_t* n_children,
                          int64_t cap_out, double* o_theta, double* o_m, double* o_v) {
  int K = (deg + 1) * (deg + 1);
  int P = 11 + 3 * K;
  (void)n_views;
  reg_key_t* keys = (reg_key_t*)malloc(sizeof(reg_key_t) * (size_t)(n_reg > 0 ? n_reg : 1));
  for (int64_t r = 0; r < n_reg; ++r) {
    keys[r].parent = r_parent[r]; keys[r].view = r_view[r]; keys[r].label = r_label[r]; keys[r].idx = r;
  }
  qsort(keys, (size_t)n_reg, sizeof(reg_key_t), reg_key_cmp);

  uint8_t* is_cand = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int64_t c = 0; c < n_cand; ++c) is_cand[cand[c]] = 1;

  /* Children of every ADAPTIVE candidate, kept in memory until the write. */
  double* kids = (double*)malloc(sizeof(double) * (size_t)P * (size_t)(n_reg > 0 ? n_reg : 1));
  int64_t* kid_start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_cand + 1));
  int64_t nk = 0, rp = 0;
  for (int64_t c = 0; c < n_cand; ++c) {
    int32_t i = cand[c];
    kid_start[c] = nk;
    while (rp < n_reg && keys[rp].parent < i) ++rp;
    int64_t r0 = rp;
    while (rp < n_reg && keys[rp].parent == i) ++rp;
    int32_t M = (int32_t)(rp - r0);
    n_children[c] = 0;
    if (count[i] == 0) { status[c] = ORC_FALLBACK; continue; }
    if (M == 0) { status[c] = ORC_RESET; continue; }
    status[c] = ORC_ADAPTIVE;
    const double* th = theta + (int64_t)i * P;
    double* pmu = (double*)malloc(sizeof(double) * 3 * (size_t)M);
    double* pR = (double*)malloc(sizeof(double) * 9 * (size_t)M);
    double* ps = (double*)malloc(sizeof(double) * 3 * (size_t)M);
    double* prgb = (double*)malloc(sizeof(double) * 3 * (size_t)M);
    for (int m = 0; m < M; ++m) {
      int64_t r = keys[r0 + m].idx;
      double ts;
      orc_child_proposal(th, &cams[r_view[r]], r_stats + 12 * r, sc->eps_t, sc->scale_floor,
                         pmu + 3 * m, pR + 9 * m, ps + 3 * m, prgb + 3 * m, &ts);
    }
    int32_t* gof = (int32_t*)malloc(sizeof(int32_t) * (size_t)M);
    double* gmu = (double*)malloc(sizeof(double) * 3 * (size_t)M);
    double* grgb = (double*)malloc(sizeof(double) * 3 * (size_t)M);
    double* gR = (double*)malloc(sizeof(double) * 9 * (size_t)M);
    double* gs = (double*)malloc(sizeof(double) * 3 * (size_t)M);
    int32_t ng = orc_merge(M, pmu, pR, ps, prgb, sc->gamma_d, sc->gamma_c, sc->scale_floor, gof,
                           gmu, grgb, gR, gs, NULL);
    ext_key_t* ek = (ext_key_t*)malloc(sizeof(ext_key_t) * (size_t)ng);
    for (int g = 0; g < ng; ++g) { ek[g].extent = gs[3 * g] * gs[3 * g + 1] * gs[3 * g + 2]; ek[g].g = g; }
    qsort(ek, (size_t)ng, sizeof(ext_key_t), ext_key_cmp);
    int32_t keep = ng < sc->n_max ? ng : sc->n_max;
    uint8_t* kept = (uint8_t*)calloc((size_t)ng, 1);
    for (int j = 0; j < keep; ++j) kept[ek[j].g] = 1;
    for (int g = 0; g < ng; ++g) {
      if (!kept[g]) continue;
      write_child(kids + nk * P, P, K, gmu + 3 * g, gR + 9 * g, gs + 3 * g, grgb + 3 * g, th[TH_LOGIT]);
      ++nk;
    }
    n_children[c] = keep;
    free(pmu); free(pR); free(ps); free(prgb); free(gof); free(gmu); free(grgb); free(gR);
    free(gs); free(ek); free(kept);
  }
  kid_start[n_cand] = nk;

  int64_t n_keep = 0;
  for (int64_t i = 0; i < n; ++i) n_keep += !is_cand[i];
  int64_t new_n = n_keep;
  for (int64_t c = 0; c < n_cand; ++c) {
    if (status[c] == ORC_RESET) new_n += 1;
    else if (status[c] == ORC_FALLBACK) new_n += 2;
    else new_n += 1 + n_children[c];
  }
  if (new_n <= cap_out && o_theta) {
    int64_t o = 0;
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) {
      while (c < n_cand && cand[c] < i) ++c;
      int candidate = (c < n_cand && cand[c] == i);
      if (candidate && status[c] != ORC_RESET) continue;
      memcpy(o_theta + o * P, theta + i * P, sizeof(double) * (size_t)P);
      if (o_m) {
        if (adam_m) memcpy(o_m + o * P, adam_m + i * P, sizeof(double) * (size_t)P);
        else memset(o_m + o * P, 0, sizeof(double) * (size_t)P);
      }
      if (o_v) {
        if (adam_v) memcpy(o_v + o * P, adam_v + i * P, sizeof(double) * (size_t)P);
        else memset(o_v + o * P, 0, sizeof(double) * (size_t)P);
      }
      ++o;
    }
    for (c = 0; c < n_cand; ++c) {
      int32_t i = cand[c];
      const double* th = theta + (int64_t)i * P;
      if (status[c] == ORC_RESET) continue;
      int64_t first = o;
      if (status[c] == ORC_FALLBACK) {
        double sp[3] = {exp(th[TH_LOGS]), exp(th[TH_LOGS + 1]), exp(th[TH_LOGS + 2])};
        double Rp[9];
        quat_to_rot(th + TH_QUAT, Rp);
        for (int ch = 0; ch < 2; ++ch) {
          double* out = o_theta + o * P;
          memcpy(out, th, sizeof(double) * (size_t)P);
          const double* z = noise + 6 * c + 3 * ch;
          double dl[3] = {sp[0] * z[0], sp[1] * z[1], sp[2] * z[2]};
          for (int r = 0; r < 3; ++r)
            out[TH_MEAN + r] = th[TH_MEAN + r] + Rp[3 * r] * dl[0] + Rp[3 * r + 1] * dl[1] + Rp[3 * r + 2] * dl[2];
          for (int r = 0; r < 3; ++r) out[TH_LOGS + r] = log(sp[r] / (sc->eta * 2.0));
          ++o;
        }
      } else {
        double* out = o_theta + o * P;
        memcpy(out, th, sizeof(double) * (size_t)P);
        out[TH_LOGIT] = logit_of(sigmoid(th[TH_LOGIT]) / (double)(n_children[c] + 1));
        ++o;
        for (int64_t k = kid_start[c]; k < kid_start[c + 1]; ++k) {
          memcpy(o_theta + o * P, kids + k * P, sizeof(double) * (size_t)P);
          ++o;
        }
      }
      for (int64_t j = first; j < o; ++j) {
        if (o_m) memset(o_m + j * P, 0, sizeof(double) * (size_t)P);
        if (o_v) memset(o_v + j * P, 0, sizeof(double) * (size_t)P);
      }
    }
  }
  free(keys);
  free(is_cand);
  free(kids);
  free(kid_start);
  return new_n;
}

/* ------------------------------------------------------------------------ */
/* Gradient of the L1 training loss (complex-step derivative of the forward)  */
/* ------------------------------------------------------------------------ */

/* Composites one pixel with Gaussian g's 9 projected outputs replaced by the
 * complex values og (the rest real); the contributor list and every branch
 * (threshold, stop, clamp) are those of the real forward. */
static void composite_c(const proj_view_t* pv, const orc_config* cfg, const double* bg,
                        const contrib_t* list, int cnt, int x, int y, int64_t g,
                        const cplx* og, cplx* col) {
  cplx T = 1.0;
  col[0] = col[1] = col[2] = 0.0;
  for (int k = 0; k < cnt; ++k) {
    if (!list[k].include) continue;
    int64_t i = list[k].id;
    cplx a;
    cplx c[3];
    if (i == g) {
      cplx dx = og[0] - x, dy = og[1] - y;
      cplx power = -0.5 * (og[2] * dx * dx + og[4] * dy * dy) - og[3] * dx * dy;
      a = og[5] * cexp(power);
      for (int ch = 0; ch < 3; ++ch) c[ch] = og[6 + ch];
    } else {
      a = list[k].alpha_raw;
      for (int ch = 0; ch < 3; ++ch) c[ch] = pv->rgb[3 * i + ch];
    }
    if (creal(a) > cfg->alpha_max) a = cfg->alpha_max;
    cplx test = T * (1.0 - a);
    if (creal(test) < cfg->t_min) break;
    for (int ch = 0; ch < 3; ++ch) col[ch] += T * a * c[ch];
    T = test;
  }
  for (int ch = 0; ch < 3; ++ch) col[ch] += T * bg[ch];
}

/* dL/dtheta for the Gaussians in sel, with L = loss_scale * sum over pixels
 * and channels of |I^ - I_gt| for one view (loss_scale = 1 / (3 W H) gives
 * the mean; sign(0) = 0). Each Gaussian's gradient collects the pixels of its
 * own box. grad is [n_sel][11 + 3K]. If mean2d_grad is not NULL it receives
 * [n_sel][2], dL with respect to the projected 2D mean (pixel units) -- the
 * image-space gradient the densification statistic of Eq. 2 accumulates. */
ORC_API void orc_grad(int64_t n, int32_t deg, const double* theta, const orc_camera* cam,
                      const orc_config* cfg, const double* bg, const float* tgt,
                      double loss_scale, int64_t n_sel, const int32_t* sel, double* grad,
                      double* mean2d_grad) {
  int P = 11 + 3 * (deg + 1) * (deg + 1);
  int W = cam->width;
  double* mean2d = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
  double* cov2d = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  double* conic = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  double* depth = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* opac = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* rgb = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  int32_t* box = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
  int32_t* rect = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
  int32_t* tiles = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  orc_project(n, deg, theta, cam, cfg, mean2d, cov2d, conic, depth, opac, rgb, NULL, box, rect, tiles);
  proj_view_t pv = {mean2d, conic, depth, opac, rgb, box, tiles};
  const double h = 1e-30;
#pragma omp parallel
  {
    contrib_t* cands = (contrib_t*)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
    contrib_t* list = (contrib_t*)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 1)
    for (int64_t si = 0; si < n_sel; ++si) {
      int64_t g = sel[si];
      double* gr = grad + si * P;
      for (int p = 0; p < P; ++p) gr[p] = 0.0;
      if (mean2d_grad) mean2d_grad[2 * si] = mean2d_grad[2 * si + 1] = 0.0;
      if (tiles[g] <= 0) continue;
      const int32_t* gb = box + 4 * g;
      /* Every Gaussian that can contribute inside g's box, depth-sorted. */
      int nc = 0;
      for (int64_t i = 0; i < n; ++i) {
        if (tiles[i] <= 0) continue;
        const int32_t* b = box + 4 * i;
        if (b[1] < gb[0] || b[0] > gb[1] || b[3] < gb[2] || b[2] > gb[3]) continue;
        contrib_t c = {depth[i], (int32_t)i, 1, 0.0};
        cands[nc++] = c;
      }
      qsort(cands, (size_t)nc, sizeof(contrib_t), contrib_cmp);
      double dL[9] = {0};
      cplx og[9];
      for (int j = 0; j < 9; ++j) og[j] = 0;
      og[0] = mean2d[2 * g]; og[1] = mean2d[2 * g + 1];
      og[2] = conic[3 * g]; og[3] = conic[3 * g + 1]; og[4] = conic[3 * g + 2];
      og[5] = opac[g];
      og[6] = rgb[3 * g]; og[7] = rgb[3 * g + 1]; og[8] = rgb[3 * g + 2];
      for (int y = gb[2]; y <= gb[3]; ++y)
        for (int x = gb[0]; x <= gb[1]; ++x) {
          int cnt = 0;
          for (int k = 0; k < nc; ++k) {
            int64_t i = cands[k].id;
            const int32_t* b = box + 4 * i;
            if (x < b[0] || x > b[1] || y < b[2] || y > b[3]) continue;
            double a = alpha_raw_at(&pv, i, x, y);
            if (a < cfg->alpha_min) continue;
            contrib_t c = {depth[i], (int32_t)i, 1, a};
            list[cnt++] = c;
          }
          pixel_out_t po;
          composite(&pv, cfg, bg, list, cnt, &po);
          /* Does g contribute before the stop? */
          double T = 1.0;
          int hit = 0;
          for (int k = 0; k < cnt; ++k) {
            double a = list[k].alpha_raw < cfg->alpha_max ? list[k].alpha_raw : cfg->alpha_max;
            if (T * (1.0 - a) < cfg->t_min) break;
            if (list[k].id == g) { hit = 1; break; }
            T *= (1.0 - a);
          }
          if (!hit) continue;
          const float* tp = tgt + 3 * ((int64_t)y * W + x);
          double sgn[3];
          for (int ch = 0; ch < 3; ++ch) {
            double d = po.rgb[ch] - (double)tp[ch];
            sgn[ch] = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
          }
          for (int j = 0; j < 9; ++j) {
            cplx oj[9];
            memcpy(oj, og, sizeof(oj));
            oj[j] += I * h;
            cplx col[3];
            composite_c(&pv, cfg, bg, list, cnt, x, y, g, oj, col);
            for (int ch = 0; ch < 3; ++ch) dL[j] += loss_scale * sgn[ch] * cimag(col[ch]) / h;
          }
        }
      if (mean2d_grad) {
        mean2d_grad[2 * si] = dL[0];
        mean2d_grad[2 * si + 1] = dL[1];
      }
      /* Jacobian of the projection by complex step. */
      cplx th[59];
      for (int p = 0; p < P; ++p) th[p] = theta[g * P + p];
      for (int p = 0; p < P; ++p) {
        th[p] += I * h;
        cplx out[9];
        double dep, cv[3];
        int cl[3];
        int vis = proj_core(cam, cfg, deg, th, out, &dep, cv, cl);
        th[p] = theta[g * P + p];
        if (!vis) continue;
        double acc = 0;
        for (int j = 0; j < 9; ++j) acc += dL[j] * cimag(out[j]) / h;
        gr[p] = acc;
      }
    }
    free(cands);
    free(list);
  }
  free(mean2d); free(cov2d); free(conic); free(depth); free(opac); free(rgb); free(box);
  free(rect); free(tiles);
}

/* ------------------------------------------------------------------------ */
/* Adam                                                                       */
/* ------------------------------------------------------------------------ */

/* One Adam step (bias-corrected) on [n][P] parameters. lr holds one rate per
 * parameter group: mean, opacity logit, log-scale, quaternion, SH DC, SH rest. */
ORC_API void orc_adam(int64_t n, int32_t P, double* theta, const double* grad, double* m, double* v,
                      int32_t step, const double* lr, double b1, double b2, double eps) {
  double bc1 = 1.0 - pow(b1, step), bc2 = 1.0 - pow(b2, step);
  for (int64_t i = 0; i < n; ++i)
    for (int p = 0; p < P; ++p) {
      int grp = p < 3 ? 0 : (p == 3 ? 1 : (p < 7 ? 2 : (p < 11 ? 3 : (p < 14 ? 4 : 5))));
      int64_t k = i * P + p;
      m[k] = b1 * m[k] + (1.0 - b1) * grad[k];
      v[k] = b2 * v[k] + (1.0 - b2) * grad[k] * grad[k];
      double mh = m[k] / bc1, vh = v[k] / bc2;
      theta[k] -= lr[grp] * mh / (sqrt(vh) + eps);
    }
}

ORC_API int32_t orc_version(void) { return 1; }
