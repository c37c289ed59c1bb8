/*
 * gftorf_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see
 * gftorf_oracle.h for what it computes and which tests pin it).
 *
 * Written for a reader checking it against the paper: no blocking, fusion or
 * reordering beyond what the method itself states.  Per pixel, the candidate
 * Gaussians (those whose tile rectangle holds the pixel's tile, the 3DGS
 * structure the paper's rasterizer inherits) are sorted front to back by view
 * depth (ties by index) and composited one by one.
 */
#include "gftorf_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double kPi = 3.14159265358979323846;
static const double kLightSpeed = 299792458.0; /* m/s */

int ora_splat_len(void) { return ORA_SP_LEN; }

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void ora_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

static int n_feat(const double* sensor) { return 2 * (int)sensor[ORA_SE_F] + 1; }
static int n_chan(const double* sensor, const double* consts) {
  const int F = (int)sensor[ORA_SE_F];
  return F * (int)sensor[ORA_SE_P] + 1 + (consts[ORA_CO_PHASOR] != 0.0 ? 2 * F : 0) +
         (consts[ORA_CO_DEPTH] != 0.0 ? 1 : 0);
}

/* ------------------------------------------------------------------------ */
/* Projection (Sec. 3 with the 3DGS EWA splatting it builds on).             */
/* Written over complex numbers so that the complex-step method gives its    */
/* exact Jacobian; the forward pass uses the real part.                      */
/* ------------------------------------------------------------------------ */

/* 2D record: u, v, conic a, b, c, opacity, features[2F+1], distance d */
#define REC_U 0
#define REC_V 1
#define REC_A 2
#define REC_B 3
#define REC_C 4
#define REC_O 5
#define REC_FEAT 6

typedef struct {
  double z;      /* view-space depth (real part) */
  double d;      /* distance to the optical centre */
  double s00, s01, s11; /* 2D covariance incl. dilation */
  double det;
} proj_aux;

/* Real spherical harmonics of degree 0..3 (orthonormal on the unit sphere),
 * Cartesian form at a unit vector, without the Condon-Shortley phase; the
 * normalisations are written out from their closed forms. */
static cplx sh_basis_c(int l, cplx x, cplx y, cplx z) {
  const double pi = kPi;
  switch (l) {
    case 0: return 0.5 * sqrt(1.0 / pi);
    case 1: return sqrt(3.0 / (4.0 * pi)) * y;
    case 2: return sqrt(3.0 / (4.0 * pi)) * z;
    case 3: return sqrt(3.0 / (4.0 * pi)) * x;
    case 4: return 0.5 * sqrt(15.0 / pi) * x * y;
    case 5: return 0.5 * sqrt(15.0 / pi) * y * z;
    case 6: return 0.25 * sqrt(5.0 / pi) * (2.0 * z * z - x * x - y * y);
    case 7: return 0.5 * sqrt(15.0 / pi) * x * z;
    case 8: return 0.25 * sqrt(15.0 / pi) * (x * x - y * y);
    case 9: return 0.25 * sqrt(35.0 / (2.0 * pi)) * y * (3.0 * x * x - y * y);
    case 10: return 0.5 * sqrt(105.0 / pi) * x * y * z;
    case 11: return 0.25 * sqrt(21.0 / (2.0 * pi)) * y * (4.0 * z * z - x * x - y * y);
    case 12: return 0.25 * sqrt(7.0 / pi) * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    case 13: return 0.25 * sqrt(21.0 / (2.0 * pi)) * x * (4.0 * z * z - x * x - y * y);
    case 14: return 0.25 * sqrt(105.0 / pi) * z * (x * x - y * y);
    case 15: return 0.25 * sqrt(35.0 / (2.0 * pi)) * x * (x * x - 3.0 * y * y);
  }
  return 0.0;
}

double ora_sh_basis(int l, double x, double y, double z) {
  return creal(sh_basis_c(l, x, y, z));
}

/* theta: mu[0..2], c1[3..5], c2[6..8], c3[9..11], scale[12..14],
 * quat[15..18] (w x y z), opacity[19], amplitude[20], delta[21..23],
 * sh[24..39]. */
static void project_complex(const cplx* th, const double* frame,
                            const double* sensor, const double* consts,
                            cplx* rec, proj_aux* aux) {
  const double t = frame[ORA_FR_TIME];
  const double* Rt = frame + ORA_FR_RT;
  const double fx = frame[ORA_FR_FX], fy = frame[ORA_FR_FY];
  const double cx = frame[ORA_FR_CX], cy = frame[ORA_FR_CY];
  const double W = frame[ORA_FR_W], H = frame[ORA_FR_H];

  /* deformation: cubic trajectory plus per-frame displacement; between two
   * timesteps t0 < t1, Eq. 7: x(t) = ((t1 - t) x(t0) + (t - t0) x(t1)) / (t1 - t0)
   * (the paper's unit-spaced integer steps, rescaled to time) */
  const double t0 = frame[ORA_FR_T0], t1 = frame[ORA_FR_T1];
  cplx x[3];
  for (int a = 0; a < 3; ++a) {
    if (t1 > t0) {
      cplx xa = th[a] + th[3 + a] * t0 + th[6 + a] * (t0 * t0) + th[9 + a] * (t0 * t0 * t0);
      cplx xb = th[a] + th[3 + a] * t1 + th[6 + a] * (t1 * t1) + th[9 + a] * (t1 * t1 * t1);
      x[a] = ((t1 - t) * xa + (t - t0) * xb) / (t1 - t0) + th[21 + a];
    } else {
      x[a] = th[a] + th[3 + a] * t + th[6 + a] * (t * t) + th[9 + a] * (t * t * t) +
             th[21 + a];
    }
  }

  /* view transform p = R x + t */
  cplx p[3];
  for (int r = 0; r < 3; ++r)
    p[r] = Rt[4 * r + 0] * x[0] + Rt[4 * r + 1] * x[1] + Rt[4 * r + 2] * x[2] +
           Rt[4 * r + 3];

  /* distance from the Gaussian centre to the optical centre o = -R^T t */
  cplx dist2 = 0;
  for (int a = 0; a < 3; ++a) {
    double o_a = -(Rt[0 * 4 + a] * Rt[3] + Rt[1 * 4 + a] * Rt[7] +
                   Rt[2 * 4 + a] * Rt[11]);
    cplx e = x[a] - o_a;
    dist2 += e * e;
  }
  cplx dist = csqrt(dist2);

  /* 3D covariance Sigma = Rq diag(s^2) Rq^T from the normalised quaternion */
  cplx qn = csqrt(th[15] * th[15] + th[16] * th[16] + th[17] * th[17] +
                  th[18] * th[18]);
  cplx w = th[15] / qn, qx = th[16] / qn, qy = th[17] / qn, qz = th[18] / qn;
  cplx Rq[9] = {
      1.0 - 2.0 * (qy * qy + qz * qz), 2.0 * (qx * qy - w * qz),
      2.0 * (qx * qz + w * qy),        2.0 * (qx * qy + w * qz),
      1.0 - 2.0 * (qx * qx + qz * qz), 2.0 * (qy * qz - w * qx),
      2.0 * (qx * qz - w * qy),        2.0 * (qy * qz + w * qx),
      1.0 - 2.0 * (qx * qx + qy * qy)};
  cplx s2[3] = {th[12] * th[12], th[13] * th[13], th[14] * th[14]};
  cplx Sig[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k) acc += Rq[3 * i + k] * s2[k] * Rq[3 * j + k];
      Sig[3 * i + j] = acc;
    }

  /* local affine approximation of the perspective projection (EWA) with the
   * 3DGS guard band on the lateral coordinates */
  cplx z = p[2];
  double limx = consts[ORA_CO_GUARD] * 0.5 * W / fx;
  double limy = consts[ORA_CO_GUARD] * 0.5 * H / fy;
  cplx txz = p[0] / z, tyz = p[1] / z;
  if (creal(txz) > limx) txz = limx;
  if (creal(txz) < -limx) txz = -limx;
  if (creal(tyz) > limy) tyz = limy;
  if (creal(tyz) < -limy) tyz = -limy;
  cplx xc = txz * z, yc = tyz * z;
  cplx J[6] = {fx / z, 0.0, -fx * xc / (z * z), 0.0, fy / z, -fy * yc / (z * z)};
  cplx M[6]; /* M = J R (2x3) */
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j)
      M[3 * i + j] = J[3 * i + 0] * Rt[0 * 4 + j] + J[3 * i + 1] * Rt[1 * 4 + j] +
                     J[3 * i + 2] * Rt[2 * 4 + j];
  cplx S2[4]; /* M Sigma M^T */
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) acc += M[3 * i + k] * Sig[3 * k + l] * M[3 * j + l];
      S2[2 * i + j] = acc;
    }
  cplx s00 = S2[0] + consts[ORA_CO_DIL];
  cplx s01 = S2[1];
  cplx s11 = S2[3] + consts[ORA_CO_DIL];
  cplx det = s00 * s11 - s01 * s01;

  rec[REC_U] = fx * p[0] / z + cx;
  rec[REC_V] = fy * p[1] / z + cy;
  rec[REC_A] = s11 / det;
  rec[REC_B] = -s01 / det;
  rec[REC_C] = s00 / det;
  rec[REC_O] = th[19];

  /* reflectivity r_k (Sec. 3, C-ToF image formation): a scalar, or view
   * dependent through up to 16 real SH coefficients evaluated at the unit
   * direction from the optical centre to the (deformed) centre, with the
   * 3DGS colour convention r = max(0, 0.5 + sum_l sh_l Y_l) */
  cplx refl = th[20];
  const int nsh = (int)consts[ORA_CO_NSH];
  if (nsh > 0) {
    cplx dir[3];
    for (int a = 0; a < 3; ++a) {
      double o_a = -(Rt[0 * 4 + a] * Rt[3] + Rt[1 * 4 + a] * Rt[7] + Rt[2 * 4 + a] * Rt[11]);
      dir[a] = (x[a] - o_a) / dist;
    }
    cplx val = 0.5;
    for (int l = 0; l < nsh; ++l) val += th[24 + l] * sh_basis_c(l, dir[0], dir[1], dir[2]);
    refl = creal(val) > 0.0 ? val : 0.0;
  }

  /* C-ToF terms (Sec. 2, Eq. 3/4): A = s r / d^2, psi_f = 4 pi d f / c */
  cplx A = sensor[ORA_SE_S] * refl / (dist * dist);
  int F = (int)sensor[ORA_SE_F];
  for (int f = 0; f < F; ++f) {
    cplx psi = 4.0 * kPi * dist * sensor[ORA_SE_FREQ + f] / kLightSpeed;
    rec[REC_FEAT + 2 * f] = A * csin(psi);
    rec[REC_FEAT + 2 * f + 1] = A * ccos(psi);
  }
  rec[REC_FEAT + 2 * F] = A;
  rec[REC_FEAT + 2 * F + 1] = dist;  /* the mean depth's d_k (Eq. 5) */

  if (aux) {
    aux->z = creal(z);
    aux->d = creal(dist);
    aux->s00 = creal(s00);
    aux->s01 = creal(s01);
    aux->s11 = creal(s11);
    aux->det = creal(det);
  }
}

static void gather_theta(int g, const double* means, const double* coeffs,
                         const double* scales, const double* quats,
                         const double* opacity, const double* amplitude,
                         const double* delta, const double* sh, cplx* th) {
  for (int a = 0; a < 3; ++a) th[a] = means[3 * g + a];
  for (int a = 0; a < 9; ++a) th[3 + a] = coeffs ? coeffs[9 * g + a] : 0.0;
  for (int a = 0; a < 3; ++a) th[12 + a] = scales[3 * g + a];
  for (int a = 0; a < 4; ++a) th[15 + a] = quats[4 * g + a];
  th[19] = opacity[g];
  th[20] = amplitude[g];
  for (int a = 0; a < 3; ++a) th[21 + a] = delta ? delta[3 * g + a] : 0.0;
  for (int l = 0; l < ORA_MAX_SH; ++l) th[24 + l] = sh ? sh[(size_t)ORA_MAX_SH * g + l] : 0.0;
}

static int clampi(double v, int lo, int hi) {
  if (!(v > lo)) return lo; /* also catches NaN */
  if (v > hi) return hi;
  return (int)v;
}

/* tile rectangle of the disc |p - (u, v)| <= r, as [x0,x1) x [y0,y1) */
static void tile_rect(double u, double v, double r, double tw, double th,
                      int tiles_x, int tiles_y, double* out) {
  out[0] = clampi(floor((u - r) / tw), 0, tiles_x);
  out[1] = clampi(floor((v - r) / th), 0, tiles_y);
  out[2] = clampi(floor((u + r) / tw) + 1.0, 0, tiles_x);
  out[3] = clampi(floor((v + r) / th) + 1.0, 0, tiles_y);
}

static int rect_empty(const double* r) { return r[0] >= r[2] || r[1] >= r[3]; }

void ora_project(int n, const double* means, const double* coeffs,
                 const double* scales, const double* quats,
                 const double* opacity, const double* amplitude,
                 const double* delta, const double* sh, const double* frame,
                 const double* sensor, const double* consts,
                 const double* eps, double* splats) {
  const int W = (int)frame[ORA_FR_W], H = (int)frame[ORA_FR_H];
  const double tw = consts[ORA_CO_TW], th_ = consts[ORA_CO_TH];
  const int tiles_x = (int)((W + tw - 1) / tw), tiles_y = (int)((H + th_ - 1) / th_);
  const int nf = n_feat(sensor);
  const double near = frame[ORA_FR_NEAR];
  const double er = eps[ORA_EPS_RECT];
#pragma omp parallel for schedule(static)
  for (int g = 0; g < n; ++g) {
    cplx th[ORA_NPARAM], rec[REC_FEAT + ORA_MAX_FEAT + 1];
    proj_aux aux;
    double* sp = splats + (size_t)g * ORA_SP_LEN;
    memset(sp, 0, sizeof(double) * ORA_SP_LEN);
    gather_theta(g, means, coeffs, scales, quats, opacity, amplitude, delta, sh, th);
    project_complex(th, frame, sensor, consts, rec, &aux);

    double u = creal(rec[REC_U]), v = creal(rec[REC_V]);
    sp[ORA_SP_U] = u;
    sp[ORA_SP_V] = v;
    sp[ORA_SP_CA] = creal(rec[REC_A]);
    sp[ORA_SP_CB] = creal(rec[REC_B]);
    sp[ORA_SP_CC] = creal(rec[REC_C]);
    sp[ORA_SP_OPA] = creal(rec[REC_O]);
    sp[ORA_SP_Z] = aux.z;
    sp[ORA_SP_D] = aux.d;
    sp[ORA_SP_AMP] = creal(rec[REC_FEAT + nf - 1]);
    for (int f = 0; f < nf; ++f) sp[ORA_SP_FEAT + f] = creal(rec[REC_FEAT + f]);

    /* cull: in front of the near plane, invertible 2D covariance */
    int in_front = aux.z > near;
    int cull_uncertain = fabs(aux.z - near) <= er * near;
    int finite = isfinite(u) && isfinite(v) && isfinite(aux.det);
    if (!finite || aux.det <= 0.0 || (!in_front && !cull_uncertain)) {
      continue; /* VIS = 0, all rects empty */
    }
    /* 3-sigma radius of the larger eigenvalue (floor 0.1 on the discriminant) */
    double mid = 0.5 * (aux.s00 + aux.s11);
    double lam = mid + sqrt(fmax(0.1, mid * mid - aux.det));
    double rr = consts[ORA_CO_SIGMA] * sqrt(lam);
    double r = ceil(rr);
    double r_lo = ceil(rr * (1.0 - er)), r_hi = ceil(rr * (1.0 + er));
    double mu = er * (fabs(u) + 1.0), mv = er * (fabs(v) + 1.0);
    double nom[4], outer[4], inner[4];
    tile_rect(u, v, r, tw, th_, tiles_x, tiles_y, nom);
    /* outer: largest rect any nearby (u, v, r) gives; inner: smallest */
    {
      double a[4], b[4];
      tile_rect(u - mu, v - mv, r_hi, tw, th_, tiles_x, tiles_y, a);
      tile_rect(u + mu, v + mv, r_hi, tw, th_, tiles_x, tiles_y, b);
      outer[0] = fmin(a[0], b[0]);
      outer[1] = fmin(a[1], b[1]);
      outer[2] = fmax(a[2], b[2]);
      outer[3] = fmax(a[3], b[3]);
      tile_rect(u - mu, v - mv, r_lo, tw, th_, tiles_x, tiles_y, a);
      tile_rect(u + mu, v + mv, r_lo, tw, th_, tiles_x, tiles_y, b);
      inner[0] = fmax(a[0], b[0]);
      inner[1] = fmax(a[1], b[1]);
      inner[2] = fmin(a[2], b[2]);
      inner[3] = fmin(a[3], b[3]);
    }
    int vis = in_front && !rect_empty(nom);
    sp[ORA_SP_VIS] = vis;
    sp[ORA_SP_RAD] = vis ? r : 0.0;
    sp[ORA_SP_UNCERT] = cull_uncertain;
    for (int k = 0; k < 4; ++k) {
      sp[ORA_SP_X0 + k] = vis ? nom[k] : 0.0;
      sp[ORA_SP_MX0 + k] = outer[k];
      sp[ORA_SP_IX0 + k] = (vis && !cull_uncertain) ? inner[k] : 0.0;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Per-pixel compositing (Eq. 4) and its backward (Eq. S3).                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int g;
  double z;
  int nominal;   /* member of the tile by the nominal rect and visible */
  int uncertain; /* membership or cull within margin */
} cand_t;

static int cmp_cand(const void* pa, const void* pb) {
  const cand_t* a = (const cand_t*)pa;
  const cand_t* b = (const cand_t*)pb;
  if (a->z < b->z) return -1;
  if (a->z > b->z) return 1;
  return (a->g > b->g) - (a->g < b->g);
}

static int in_rect(const double* r, int tx, int ty) {
  return tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3];
}

/* all Gaussians that may cover tile (tx, ty), sorted by (depth, index) */
static int collect_candidates(int n, const double* splats, int tx, int ty,
                              cand_t* out) {
  int m = 0;
  for (int g = 0; g < n; ++g) {
    const double* sp = splats + (size_t)g * ORA_SP_LEN;
    if (!in_rect(sp + ORA_SP_MX0, tx, ty)) continue;
    cand_t c;
    c.g = g;
    c.z = sp[ORA_SP_Z];
    c.nominal = sp[ORA_SP_VIS] != 0.0 && in_rect(sp + ORA_SP_X0, tx, ty);
    c.uncertain = sp[ORA_SP_UNCERT] != 0.0 || !in_rect(sp + ORA_SP_IX0, tx, ty);
    out[m++] = c;
  }
  qsort(out, (size_t)m, sizeof(cand_t), cmp_cand);
  return m;
}

/* one composited Gaussian of a pixel, kept for the backward walk */
typedef struct {
  int g;
  double alpha, T, G, dx, dy;
  int clamped;
} step_t;

/* A decision of the walk that a single-precision implementation may take
 * the other way, because the oracle's value lies within the margin of the
 * threshold: its kind (an ORA_AMB_* bit) and the Gaussian it concerns (for
 * ORA_AMB_ORDER also g2, the composited Gaussian of nearly equal depth just
 * before it).  A walk can be re-run with a set of them forced the other way. */
typedef struct {
  int g, kind, g2;
} flip_t;

static int is_forced(const flip_t* f, int nf, int g, int kind) {
  for (int i = 0; i < nf; ++i)
    if (f[i].g == g && f[i].kind == kind) return 1;
  return 0;
}

/* record a near-threshold decision (not already forced in this walk) */
static void note_flip(flip_t* out, int* nout, int max_out, const flip_t* force, int nforce,
                      int g, int kind, int g2) {
  if (!out || is_forced(force, nforce, g, kind)) return;
  for (int i = 0; i < *nout; ++i)
    if (out[i].g == g && out[i].kind == kind) return;
  if (*nout < max_out) {
    out[*nout].g = g;
    out[*nout].kind = kind;
    out[*nout].g2 = g2;
    ++*nout;
  }
}

/* Front-to-back walk of one pixel.  Returns the number of composited
 * Gaussians (steps[] filled if non-NULL), the accumulators acc[2F+1]
 * (sum alpha T^2 feature), acc[2F+1] = sum alpha T d (mean depth, one-way T)
 * and the final one-way transmittance.
 * force[nforce]: decisions taken the other way in this walk -- a tile
 * membership (include a Gaussian outside the nominal rectangle or drop one
 * inside it), the power > 0 skip, the alpha_min skip, the T_min stop, or the
 * order of two composited Gaussians of nearly equal depth (swapped).
 * near[*nnear] (if non-NULL): the decisions of this walk within margin of
 * their thresholds, other than the forced ones. */
static int composite_walk(const double* splats, const cand_t* cand, int m,
                          double px, double py, const double* sensor,
                          const double* consts, const double* eps,
                          const flip_t* force, int nforce, flip_t* near, int* nnear,
                          int max_near, double* acc, double* T_out, int* ambig,
                          step_t* steps) {
  const int nf = n_feat(sensor);
  const double amax = consts[ORA_CO_AMAX], amin = consts[ORA_CO_AMIN];
  const double tmin = consts[ORA_CO_TMIN];
  double T = 1.0;
  int k = 0, flags = 0;
  double prev_z = -INFINITY;
  int prev_g = -1;
  /* forced order swaps: positions of the two Gaussians exchange */
  int swap_a[8], swap_b[8], nswap = 0;
  for (int i = 0; i < nforce && nswap < 8; ++i) {
    if (force[i].kind != ORA_AMB_ORDER) continue;
    int pa = -1, pb = -1;
    for (int j = 0; j < m; ++j) {
      if (cand[j].g == force[i].g2) pa = j;
      if (cand[j].g == force[i].g) pb = j;
    }
    if (pa >= 0 && pb >= 0) {
      swap_a[nswap] = pa;
      swap_b[nswap] = pb;
      ++nswap;
    }
  }
  if (nnear) *nnear = 0;
  for (int f = 0; f <= nf; ++f) acc[f] = 0.0;
  for (int i0 = 0; i0 < m; ++i0) {
    int i = i0;
    for (int q = 0; q < nswap; ++q) {
      if (i0 == swap_a[q]) i = swap_b[q];
      else if (i0 == swap_b[q]) i = swap_a[q];
    }
    const int g = cand[i].g;
#define ORA_POS(j0, jout)                                \
  do {                                                   \
    jout = (j0);                                         \
    for (int q_ = 0; q_ < nswap; ++q_) {                 \
      if ((j0) == swap_a[q_]) jout = swap_b[q_];         \
      else if ((j0) == swap_b[q_]) jout = swap_a[q_];    \
    }                                                    \
  } while (0)
    const double* sp = splats + (size_t)g * ORA_SP_LEN;
    double dx = sp[ORA_SP_U] - px, dy = sp[ORA_SP_V] - py;
    double a = sp[ORA_SP_CA], b = sp[ORA_SP_CB], c = sp[ORA_SP_CC];
    double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
    double mag = 0.5 * (fabs(a) * dx * dx + fabs(c) * dy * dy) + fabs(b * dx * dy);
    double G = exp(power);
    double oG = sp[ORA_SP_OPA] * G;
    double alpha = fmin(amax, oG);
    int would = alpha >= amin * (1.0 - eps[ORA_EPS_ALPHA]);
    int member = cand[i].nominal;
    if (!member) {
      if (would) {
        flags |= ORA_AMB_RECT;
        note_flip(near, nnear, max_near, force, nforce, g, ORA_AMB_RECT, -1);
      }
      if (!is_forced(force, nforce, g, ORA_AMB_RECT)) continue;
    } else if (is_forced(force, nforce, g, ORA_AMB_RECT)) {
      continue;
    }
    if (would && fabs(power) <= eps[ORA_EPS_ALPHA] * mag) {
      flags |= ORA_AMB_POWER;
      note_flip(near, nnear, max_near, force, nforce, g, ORA_AMB_POWER, -1);
    }
    if ((power > 0.0) != is_forced(force, nforce, g, ORA_AMB_POWER)) continue;
    if (fabs(alpha - amin) <= eps[ORA_EPS_ALPHA] * amin) {
      flags |= ORA_AMB_ALPHA_MIN;
      note_flip(near, nnear, max_near, force, nforce, g, ORA_AMB_ALPHA_MIN, -1);
    }
    if ((alpha < amin) != is_forced(force, nforce, g, ORA_AMB_ALPHA_MIN)) continue;
    if (fabs(oG - amax) <= eps[ORA_EPS_ALPHA] * amax) flags |= ORA_AMB_CLAMP;
    if (member && cand[i].uncertain) {
      flags |= ORA_AMB_RECT;
      note_flip(near, nnear, max_near, force, nforce, g, ORA_AMB_RECT, -1);
    }
    if (fabs(cand[i].z - prev_z) <= eps[ORA_EPS_Z] * fabs(cand[i].z)) {
      flags |= ORA_AMB_ORDER;
      note_flip(near, nnear, max_near, force, nforce, g, ORA_AMB_ORDER, prev_g);
    }
    prev_z = cand[i].z;
    prev_g = g;
    double t_next = T * (1.0 - alpha);
    if (fabs(t_next - tmin) <= eps[ORA_EPS_T] * (double)(k + 4) * tmin) {
      flags |= ORA_AMB_TMIN;
      note_flip(near, nnear, max_near, force, nforce, g, ORA_AMB_TMIN, -1);
    }
    /* early stop; this Gaussian is not composited */
    if ((t_next < tmin) != is_forced(force, nforce, g, ORA_AMB_TMIN)) {
      /* Gaussians of nearly equal depth just behind the stopping one: single
       * precision may order one of them first and composite it before
       * stopping, so each that could composite here is an order decision
       * (the alternative swaps the two) */
      for (int j0 = i0 + 1; j0 < m; ++j0) {
        int j;
        ORA_POS(j0, j);
        if (cand[j].z - cand[i].z > eps[ORA_EPS_Z] * fabs(cand[j].z)) break;
        if (!cand[j].nominal) continue;
        const double* sj = splats + (size_t)cand[j].g * ORA_SP_LEN;
        const double ex = sj[ORA_SP_U] - px, ey = sj[ORA_SP_V] - py;
        const double pw = -0.5 * (sj[ORA_SP_CA] * ex * ex + sj[ORA_SP_CC] * ey * ey) -
                          sj[ORA_SP_CB] * ex * ey;
        const double aj = fmin(amax, sj[ORA_SP_OPA] * exp(pw));
        if (pw > 0.0 || aj < amin * (1.0 - eps[ORA_EPS_ALPHA])) continue;
        flags |= ORA_AMB_ORDER;
        note_flip(near, nnear, max_near, force, nforce, cand[j].g, ORA_AMB_ORDER, g);
      }
      break;
    }
    double w = alpha * T * T;  /* squared transmittance: round trip */
    for (int f = 0; f < nf; ++f) acc[f] += w * sp[ORA_SP_FEAT + f];
    acc[nf] += alpha * T * sp[ORA_SP_D]; /* Eq. 5: one-way transmittance */
    if (steps) {
      steps[k].g = g;
      steps[k].alpha = alpha;
      steps[k].T = T;
      steps[k].G = G;
      steps[k].dx = dx;
      steps[k].dy = dy;
      steps[k].clamped = oG >= amax;
    }
    T = t_next;
    ++k;
  }
#undef ORA_POS
  *T_out = T;
  if (ambig) *ambig = flags;
  return k;
}

static int composite_pixel(const double* splats, const cand_t* cand, int m,
                           double px, double py, const double* sensor,
                           const double* consts, const double* eps,
                           double* acc, double* T_out, int* ambig,
                           step_t* steps) {
  return composite_walk(splats, cand, m, px, py, sensor, consts, eps, NULL, 0, NULL, NULL, 0,
                        acc, T_out, ambig, steps);
}

/* Every result the walk of pixel (px, py) takes when single precision
 * decides some of its near-threshold decisions the other way: the nominal
 * walk first, then walks with one, two or three of them forced the other way
 * (breadth first; each walk's own near-threshold decisions extend the
 * search, since a flipped decision changes T for the rest of the walk).
 * At most max_out distinct results; acc_out[max_out][2F+2], T_out[max_out].
 * Returns the number of distinct results; *capped = 1 if the search stopped
 * at max_out. */
#define ORA_ALT_DEPTH 3
static int pixel_alternatives(const double* splats, const cand_t* cand, int m, double px,
                              double py, const double* sensor, const double* consts,
                              const double* eps, int max_out, double* acc_out, double* T_out,
                              int* capped) {
  enum { kMaxSets = 64, kMaxNear = 16 };
  flip_t sets[kMaxSets][ORA_ALT_DEPTH];
  int setn[kMaxSets];
  int nsets = 1;
  setn[0] = 0;
  int nout = 0;
  *capped = 0;
  const int stride = ORA_MAX_FEAT + 1;
  for (int s = 0; s < nsets; ++s) {
    if (nout == max_out) {
      *capped = 1;
      break;
    }
    flip_t near[kMaxNear];
    int nnear = 0;
    double* acc = acc_out + (size_t)nout * stride;
    for (int f = 0; f < stride; ++f) acc[f] = 0.0; /* the walk fills 2F+2 of them */
    composite_walk(splats, cand, m, px, py, sensor, consts, eps, sets[s], setn[s], near, &nnear,
                   kMaxNear, acc, T_out + nout, NULL, NULL);
    /* keep the result unless an earlier walk gave exactly the same one (two
     * swaps of the same pair restore the order) */
    int same = 0;
    for (int o = 0; o < nout && !same; ++o) {
      same = T_out[o] == T_out[nout];
      for (int f = 0; f < stride && same; ++f) same = acc_out[(size_t)o * stride + f] == acc[f];
    }
    if (!same) ++nout;
    if (setn[s] == ORA_ALT_DEPTH) continue;
    for (int a = 0; a < nnear; ++a) {
      /* the set sets[s] + near[a], unless an equal set is queued already */
      int dup = 0;
      for (int t = 0; t < nsets && !dup; ++t) {
        if (setn[t] != setn[s] + 1) continue;
        int all = 1;
        for (int u = 0; u < setn[t] && all; ++u) {
          const flip_t* x = &sets[t][u];
          int found = x->g == near[a].g && x->kind == near[a].kind;
          for (int v = 0; v < setn[s] && !found; ++v)
            found = x->g == sets[s][v].g && x->kind == sets[s][v].kind;
          all = found;
        }
        dup = all;
      }
      if (dup) continue;
      if (nsets == kMaxSets) {
        *capped = 1;
        break;
      }
      for (int u = 0; u < setn[s]; ++u) sets[nsets][u] = sets[s][u];
      sets[nsets][setn[s]] = near[a];
      setn[nsets] = setn[s] + 1;
      ++nsets;
    }
  }
  return nout;
}

/* raw samples from the accumulators: Q_fj = cos(phi_j) S_f + sin(phi_j) C_f
 * + bg_fj T, i.e. sum w A sin(psi + phi_j) + bg T; ambient = I + bg_amb T;
 * phasor (Eq. 3) = 2 (C_f + i S_f) + bg T; mean depth (Eq. 5) as summed */
static void samples_from_acc(const double* acc, double T, const double* bg,
                             const double* frame, const double* sensor,
                             const double* consts, double* q, size_t stride) {
  const int F = (int)sensor[ORA_SE_F], P = (int)sensor[ORA_SE_P];
  for (int f = 0; f < F; ++f)
    for (int j = 0; j < P; ++j) {
      double phi = sensor[ORA_SE_OFF + j] + frame[ORA_FR_PHASE];
      q[(size_t)(f * P + j) * stride] =
          cos(phi) * acc[2 * f] + sin(phi) * acc[2 * f + 1] + bg[f * P + j] * T;
    }
  int c = F * P;
  q[(size_t)c * stride] = acc[2 * F] + bg[c] * T;
  ++c;
  if (consts[ORA_CO_PHASOR] != 0.0)
    for (int f = 0; f < F; ++f, c += 2) {
      q[(size_t)c * stride] = 2.0 * acc[2 * f + 1] + bg[c] * T;
      q[(size_t)(c + 1) * stride] = 2.0 * acc[2 * f] + bg[c + 1] * T;
    }
  if (consts[ORA_CO_DEPTH] != 0.0) q[(size_t)c * stride] = acc[2 * F + 1];
}

static int max_candidates(int n) { return n > 0 ? n : 1; }

void ora_render_pixels(int n, const double* splats, const double* frame,
                       const double* sensor, const double* consts,
                       const double* bg, const double* eps, int npix,
                       const int32_t* pix, double* out, double* tfinal,
                       int32_t* ambig, int32_t* ncontrib) {
  const int C = n_chan(sensor, consts);
  const int tw = (int)consts[ORA_CO_TW], th = (int)consts[ORA_CO_TH];
#pragma omp parallel
  {
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)max_candidates(n));
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < npix; ++i) {
      int x = pix[2 * i], y = pix[2 * i + 1];
      int m = collect_candidates(n, splats, x / tw, y / th, cand);
      double acc[ORA_MAX_FEAT + 1], T;
      int flags = 0;
      int k = composite_pixel(splats, cand, m, x + 0.5, y + 0.5, sensor, consts,
                              eps, acc, &T, &flags, NULL);
      samples_from_acc(acc, T, bg, frame, sensor, consts, out + (size_t)i * C, 1);
      if (tfinal) tfinal[i] = T;
      if (ambig) ambig[i] = flags;
      if (ncontrib) ncontrib[i] = k;
    }
    free(cand);
  }
}

int ora_pixel_steps(int n, const double* splats, const double* sensor,
                    const double* consts, const double* eps, int x, int y,
                    int max_steps, double* alpha, double* trans, double* tfinal) {
  const int tw = (int)consts[ORA_CO_TW], th = (int)consts[ORA_CO_TH];
  cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)max_candidates(n));
  step_t* steps = (step_t*)malloc(sizeof(step_t) * (size_t)max_candidates(n));
  int m = collect_candidates(n, splats, x / tw, y / th, cand);
  double acc[ORA_MAX_FEAT + 1], T;
  int flags = 0;
  int k = composite_pixel(splats, cand, m, x + 0.5, y + 0.5, sensor, consts, eps, acc, &T,
                          &flags, steps);
  for (int i = 0; i < k && i < max_steps; ++i) {
    alpha[i] = steps[i].alpha;
    trans[i] = steps[i].T;
  }
  *tfinal = T;
  free(steps);
  free(cand);
  return k;
}

void ora_render_frame(int n, const double* splats, const double* frame,
                      const double* sensor, const double* consts,
                      const double* bg, const double* eps, double* out,
                      double* tfinal, int32_t* ambig, int32_t* ncontrib) {
  const int W = (int)frame[ORA_FR_W], H = (int)frame[ORA_FR_H];
  const int tw = (int)consts[ORA_CO_TW], th = (int)consts[ORA_CO_TH];
  const int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
  const size_t HW = (size_t)W * H;
#pragma omp parallel
  {
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)max_candidates(n));
#pragma omp for schedule(dynamic, 1)
    for (int tile = 0; tile < tiles_x * tiles_y; ++tile) {
      int tx = tile % tiles_x, ty = tile / tiles_x;
      /* the candidate set and its order are the same for every pixel of a
       * tile, so they are gathered once per tile */
      int m = collect_candidates(n, splats, tx, ty, cand);
      for (int y = ty * th; y < (ty + 1) * th && y < H; ++y)
        for (int x = tx * tw; x < (tx + 1) * tw && x < W; ++x) {
          double acc[ORA_MAX_FEAT + 1], T;
          int flags = 0;
          int k = composite_pixel(splats, cand, m, x + 0.5, y + 0.5, sensor,
                                  consts, eps, acc, &T, &flags, NULL);
          size_t p = (size_t)y * W + x;
          samples_from_acc(acc, T, bg, frame, sensor, consts, out + p, HW);
          if (tfinal) tfinal[p] = T;
          if (ambig) ambig[p] = flags;
          if (ncontrib) ncontrib[p] = k;
        }
    }
    free(cand);
  }
}

int64_t ora_render_tiles(int n, const double* splats, const double* frame,
                         const double* sensor, const double* consts, const double* bg,
                         const double* eps, int ntiles, const int32_t* tiles, double* out,
                         double* tfinal, int32_t* ambig, int32_t* pix, int max_alt,
                         int64_t alt_cap, double* alt_out, int64_t* alt_pix,
                         int64_t* n_alt, int64_t* n_capped) {
  const int W = (int)frame[ORA_FR_W], H = (int)frame[ORA_FR_H];
  const int tw = (int)consts[ORA_CO_TW], th = (int)consts[ORA_CO_TH];
  const int C = n_chan(sensor, consts);
  const int value_flags = ORA_AMB_ALPHA_MIN | ORA_AMB_TMIN | ORA_AMB_ORDER | ORA_AMB_RECT |
                          ORA_AMB_POWER;
  /* pixel offsets of the tiles (tile by tile, row-major, inside the image) */
  int64_t* first = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ntiles + 1));
  first[0] = 0;
  for (int t = 0; t < ntiles; ++t) {
    const int x0 = tiles[2 * t] * tw, y0 = tiles[2 * t + 1] * th;
    const int wx = x0 >= W ? 0 : (x0 + tw <= W ? tw : W - x0);
    const int wy = y0 >= H ? 0 : (y0 + th <= H ? th : H - y0);
    first[t + 1] = first[t] + (int64_t)wx * wy;
  }
  int64_t next_alt = 0, capped_px = 0;
  const int stride = ORA_MAX_FEAT + 1;
#pragma omp parallel
  {
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)max_candidates(n));
    double* accs = (double*)malloc(sizeof(double) * (size_t)(max_alt > 0 ? max_alt : 1) * stride);
    double* Ts = (double*)malloc(sizeof(double) * (size_t)(max_alt > 0 ? max_alt : 1));
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < ntiles; ++t) {
      const int tx = tiles[2 * t], ty = tiles[2 * t + 1];
      const int m = collect_candidates(n, splats, tx, ty, cand);
      int64_t p = first[t];
      for (int y = ty * th; y < (ty + 1) * th && y < H; ++y)
        for (int x = tx * tw; x < (tx + 1) * tw && x < W; ++x, ++p) {
          double acc[ORA_MAX_FEAT + 1], T;
          int flags = 0;
          composite_pixel(splats, cand, m, x + 0.5, y + 0.5, sensor, consts, eps, acc, &T,
                          &flags, NULL);
          samples_from_acc(acc, T, bg, frame, sensor, consts, out + (size_t)p * C, 1);
          tfinal[p] = T;
          ambig[p] = flags;
          pix[2 * p] = x;
          pix[2 * p + 1] = y;
          if (max_alt <= 1 || !(flags & value_flags)) continue;
          int capped = 0;
          const int k = pixel_alternatives(splats, cand, m, x + 0.5, y + 0.5, sensor, consts,
                                           eps, max_alt, accs, Ts, &capped);
          int64_t at;
#pragma omp atomic capture
          { at = next_alt; next_alt += k; }
          if (capped) {
#pragma omp atomic
            ++capped_px;
          }
          for (int i = 0; i < k; ++i) {
            if (at + i >= alt_cap) break;
            samples_from_acc(accs + (size_t)i * stride, Ts[i], bg, frame, sensor, consts,
                             alt_out + (size_t)(at + i) * C, 1);
            alt_pix[at + i] = p;
          }
        }
    }
    free(Ts);
    free(accs);
    free(cand);
  }
  *n_alt = next_alt;
  *n_capped = capped_px;
  const int64_t total = first[ntiles];
  free(first);
  return total;
}

static void atomic_add(double* p, double v) {
#pragma omp atomic
  *p += v;
}

void ora_backward_2d(int n, const double* splats, const double* frame,
                     const double* sensor, const double* consts,
                     const double* bg, const double* dout, double* g2d,
                     double* dbg) {
  const int W = (int)frame[ORA_FR_W], H = (int)frame[ORA_FR_H];
  const int tw = (int)consts[ORA_CO_TW], th = (int)consts[ORA_CO_TH];
  const int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
  const int F = (int)sensor[ORA_SE_F], P = (int)sensor[ORA_SE_P];
  const int C = n_chan(sensor, consts), nf = 2 * F + 1, stride = 7 + nf;
  const int phasor = consts[ORA_CO_PHASOR] != 0.0, depth = consts[ORA_CO_DEPTH] != 0.0;
  const size_t HW = (size_t)W * H;
  const double zero_eps[ORA_EPS_LEN] = {0, 0, 0, 0};
#pragma omp parallel
  {
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)max_candidates(n));
    step_t* steps = (step_t*)malloc(sizeof(step_t) * (size_t)max_candidates(n));
#pragma omp for schedule(dynamic, 1)
    for (int tile = 0; tile < tiles_x * tiles_y; ++tile) {
      int tx = tile % tiles_x, ty = tile / tiles_x;
      int m = -1;
      for (int y = ty * th; y < (ty + 1) * th && y < H; ++y)
        for (int x = tx * tw; x < (tx + 1) * tw && x < W; ++x) {
          size_t p = (size_t)y * W + x;
          int any = 0;
          for (int c = 0; c < C; ++c) any |= dout[c * HW + p] != 0.0;
          if (!any) continue;
          if (m < 0) m = collect_candidates(n, splats, tx, ty, cand);
          double acc_fwd[ORA_MAX_FEAT + 1], Tf;
          int K = composite_pixel(splats, cand, m, x + 0.5, y + 0.5, sensor,
                                  consts, zero_eps, acc_fwd, &Tf, NULL, steps);
          /* dL/d(accumulator): fold the raw-sample gradients (Q is linear
           * in S_f, C_f, I and T_final) */
          double gacc[ORA_MAX_FEAT] = {0};
          double gT = 0.0;
          for (int f = 0; f < F; ++f)
            for (int j = 0; j < P; ++j) {
              double gq = dout[(size_t)(f * P + j) * HW + p];
              double phi = sensor[ORA_SE_OFF + j] + frame[ORA_FR_PHASE];
              gacc[2 * f] += cos(phi) * gq;
              gacc[2 * f + 1] += sin(phi) * gq;
              gT += bg[f * P + j] * gq;
            }
          gacc[2 * F] = dout[(size_t)(F * P) * HW + p];
          gT += bg[F * P] * gacc[2 * F];
          int c = F * P + 1;
          if (phasor)
            for (int f = 0; f < F; ++f, c += 2) {  /* Re = 2 C_f, Im = 2 S_f */
              double gre = dout[(size_t)c * HW + p], gim = dout[(size_t)(c + 1) * HW + p];
              gacc[2 * f + 1] += 2.0 * gre;
              gacc[2 * f] += 2.0 * gim;
              gT += bg[c] * gre + bg[c + 1] * gim;
            }
          const double gD = depth ? dout[(size_t)c * HW + p] : 0.0;
          if (dbg)
            for (int cc = 0; cc < C; ++cc) {
              if (depth && cc == C - 1) continue; /* Eq. 5 has no background */
              atomic_add(&dbg[cc], Tf * dout[cc * HW + p]);
            }

          /* back to front: Eq. S3 with squared transmittance,
           * dq/dalpha_k = T_k^2 (q_k + 2 (alpha_k - 1) acc_k),
           * acc_{k-1} = alpha_k q_k + (1 - alpha_k)^2 acc_k, acc_last = 0;
           * plus the background term d(bg T_N)/dalpha_k = -bg T_N/(1-alpha_k) */
          double acc[ORA_MAX_FEAT] = {0};
          double accD = 0.0; /* one-way recursion of the mean depth */
          for (int k = K - 1; k >= 0; --k) {
            const step_t* s = &steps[k];
            const double* sp = splats + (size_t)s->g * ORA_SP_LEN;
            double* gg = g2d + (size_t)s->g * stride;
            double a = s->alpha, T2 = s->T * s->T;
            double dL_dalpha = -gT * Tf / (1.0 - a);
            for (int f = 0; f < nf; ++f) {
              double q = sp[ORA_SP_FEAT + f];
              dL_dalpha += gacc[f] * T2 * (q + 2.0 * (a - 1.0) * acc[f]);
              atomic_add(&gg[6 + f], gacc[f] * a * T2);
              acc[f] = a * q + (1.0 - a) * (1.0 - a) * acc[f];
            }
            if (depth) {
              /* d D / d alpha_k = T_k (d_k - accD_k), accD_{k-1} = alpha_k d_k
               * + (1 - alpha_k) accD_k (3DGS recursion, one-way T) */
              const double d = sp[ORA_SP_D];
              dL_dalpha += gD * s->T * (d - accD);
              atomic_add(&gg[6 + nf], gD * a * s->T);
              accD = a * d + (1.0 - a) * accD;
            }
            if (s->clamped) continue; /* alpha = alpha_max does not vary */
            /* alpha = o G, G = exp(power) */
            atomic_add(&gg[REC_O], dL_dalpha * s->G);
            double dL_dpow = dL_dalpha * a;
            double ca = sp[ORA_SP_CA], cb = sp[ORA_SP_CB], cc = sp[ORA_SP_CC];
            atomic_add(&gg[REC_U], dL_dpow * -(ca * s->dx + cb * s->dy));
            atomic_add(&gg[REC_V], dL_dpow * -(cc * s->dy + cb * s->dx));
            atomic_add(&gg[REC_A], dL_dpow * -0.5 * s->dx * s->dx);
            atomic_add(&gg[REC_B], dL_dpow * -s->dx * s->dy);
            atomic_add(&gg[REC_C], dL_dpow * -0.5 * s->dy * s->dy);
          }
        }
    }
    free(steps);
    free(cand);
  }
}

void ora_backward_params(int n, const double* means, const double* coeffs,
                         const double* scales, const double* quats,
                         const double* opacity, const double* amplitude,
                         const double* delta, const double* sh, const double* frame,
                         const double* sensor, const double* consts,
                         const double* splats, const double* g2d,
                         double* grads) {
  const int nf = n_feat(sensor), stride = 7 + nf;
  const double h = 1e-30; /* complex step */
#pragma omp parallel for schedule(dynamic, 64)
  for (int g = 0; g < n; ++g) {
    const double* gg = g2d + (size_t)g * stride;
    int any = 0;
    for (int r = 0; r < stride; ++r) any |= gg[r] != 0.0;
    if (!any || splats[(size_t)g * ORA_SP_LEN + ORA_SP_VIS] == 0.0) continue;
    cplx th[ORA_NPARAM], rec[REC_FEAT + ORA_MAX_FEAT + 1];
    gather_theta(g, means, coeffs, scales, quats, opacity, amplitude, delta, sh, th);
    for (int i = 0; i < ORA_NPARAM; ++i) {
      cplx saved = th[i];
      th[i] = creal(saved) + I * h;
      project_complex(th, frame, sensor, consts, rec, NULL);
      th[i] = saved;
      double s = 0.0;
      for (int r = 0; r < stride; ++r) s += gg[r] * cimag(rec[r]) / h;
      grads[(size_t)g * ORA_NPARAM + i] += s;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Binning contract (integer work; FP32 decisions)                          */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t key;
  uint32_t value;
} pair_t;

static int cmp_pair(const void* pa, const void* pb) {
  const pair_t* a = (const pair_t*)pa;
  const pair_t* b = (const pair_t*)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return (a->value > b->value) - (a->value < b->value);
}

static int clamp_tile_f32(float v, int hi) {
  if (!(v > 0.0f)) return 0;
  if (v > (float)hi) return hi;
  return (int)v;
}

int64_t ora_bin_f32(int n, int frames, const float* u, const float* v,
                    const int32_t* radius, const float* z, int width,
                    int height, int tile_w, int tile_h, int64_t capacity,
                    uint64_t* keys, uint32_t* values, uint32_t* ranges) {
  const int tiles_x = (width + tile_w - 1) / tile_w;
  const int tiles_y = (height + tile_h - 1) / tile_h;
  const int64_t tiles = (int64_t)tiles_x * tiles_y;
  const float tw = (float)tile_w, th = (float)tile_h;
  int64_t m = 0;
  pair_t* pairs = NULL;
  for (int pass = 0; pass < 2; ++pass) {
    m = 0;
    for (int b = 0; b < frames; ++b)
      for (int g = 0; g < n; ++g) {
        size_t i = (size_t)b * n + g;
        if (radius[i] <= 0) continue;
        float r = (float)radius[i];
        volatile float lo_x = u[i] - r, hi_x = u[i] + r; /* single rounding */
        volatile float lo_y = v[i] - r, hi_y = v[i] + r;
        int x0 = clamp_tile_f32(floorf(lo_x / tw), tiles_x);
        int x1 = clamp_tile_f32(floorf(hi_x / tw) + 1.0f, tiles_x);
        int y0 = clamp_tile_f32(floorf(lo_y / th), tiles_y);
        int y1 = clamp_tile_f32(floorf(hi_y / th) + 1.0f, tiles_y);
        uint32_t zb;
        memcpy(&zb, &z[i], 4);
        for (int ty = y0; ty < y1; ++ty)
          for (int tx = x0; tx < x1; ++tx) {
            if (pass == 1) {
              uint64_t tile = (uint64_t)b * tiles + (uint64_t)ty * tiles_x + tx;
              pairs[m].key = (tile << 32) | zb;
              pairs[m].value = (uint32_t)g;
            }
            ++m;
          }
      }
    if (pass == 0) {
      if (m > capacity) return -1;
      pairs = (pair_t*)malloc(sizeof(pair_t) * (size_t)(m > 0 ? m : 1));
    }
  }
  qsort(pairs, (size_t)m, sizeof(pair_t), cmp_pair);
  /* ranges: [first index of the tile, first index past it); an empty tile
   * gets [k, k) with k the number of instances in the tiles before it */
  int64_t i = 0;
  for (int64_t t = 0; t < tiles * frames; ++t) {
    ranges[2 * t] = (uint32_t)i;
    while (i < m && (int64_t)(pairs[i].key >> 32) == t) ++i;
    ranges[2 * t + 1] = (uint32_t)i;
  }
  for (int64_t k = 0; k < m; ++k) {
    keys[k] = pairs[k].key;
    values[k] = pairs[k].value;
  }
  free(pairs);
  return m;
}
