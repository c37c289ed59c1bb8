/*
 * gftorf_oracle.h -- plain FP64 CPU oracle for differentiable raw C-ToF
 * Gaussian splatting ("Time of the Flight of the Gaussians", arXiv 2505.05356).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, helper, table or constant with the CUDA path.
 *
 * What it computes (all in double precision):
 *   - time-varying Gaussian positions x_k(t) = mu + c1 t + c2 t^2 + c3 t^3
 *     (+ an optional per-frame displacement), i.e. the deformation step that
 *     stands in for the paper's MLP offsets (Sec. 4 "Pipeline"), optionally
 *     interpolated linearly between two timesteps (Eq. 7);
 *   - EWA projection of each 3D Gaussian to a 2D conic (the 3DGS convention
 *     the paper builds on, Sec. 3 "GS image formation model");
 *   - the raw C-ToF quad formation of Eq. 4 (T_k squared for the round trip,
 *     amplitude s r_k / d_k^2, phase psi_k = 4 pi d_k f / c), generalised to
 *     arbitrary phase offsets as sin(psi_k + phi_j) (Sec. 2, the Q_phi model),
 *     plus an ambient channel sum_k alpha_k T_k^2 A_k + bg T_N;
 *   - its gradient: the squared-transmittance opacity recursion of Eq. S3,
 *     and an exact (complex-step) Jacobian of the projection.
 *
 * Parity status: every function here is pinned by tests under tests/
 * (closed forms, brute force, central finite differences) except the
 * 3DGS screen-space conventions (dilation 0.3, guard band 1.3, 3-sigma radius
 * with the 0.1 eigenvalue floor): the paper inherits them without stating
 * them, so their values are "parity unpinned" -- pinned only by oracle/CUDA
 * agreement.
 *
 * Packed argument layouts (double arrays) are given by the enums below.
 */
#ifndef GFTORF_ORACLE_H
#define GFTORF_ORACLE_H

#include <stdint.h>

#define ORA_MAX_F 4
#define ORA_MAX_P 8
#define ORA_MAX_FEAT (2 * ORA_MAX_F + 1)
#define ORA_MAX_SH 16
/* mu[3] c[9] scale[3] quat[4] opacity amplitude delta[3] sh[16] */
#define ORA_NPARAM (24 + ORA_MAX_SH)

/* one frame: camera + time */
enum {
  ORA_FR_W = 0, ORA_FR_H, ORA_FR_FX, ORA_FR_FY, ORA_FR_CX, ORA_FR_CY,
  ORA_FR_RT,               /* 12 values, row-major 3x4 world->camera [R | t] */
  ORA_FR_NEAR = ORA_FR_RT + 12,
  ORA_FR_TIME,
  ORA_FR_PHASE,  /* added to every sensor phase offset in this frame: an
                    asynchronously captured raw frame (Sec. 3) samples its
                    own offset at its own time */
  ORA_FR_T0,     /* Eq. 7: with T0 < T1 the positions at TIME are the linear */
  ORA_FR_T1,     /* interpolation of those at the timesteps T0 and T1;
                    T0 == T1: positions at TIME directly */
  ORA_FR_LEN
};
/* sensor */
enum {
  ORA_SE_F = 0, ORA_SE_FREQ,              /* ORA_MAX_F frequencies in Hz */
  ORA_SE_P = ORA_SE_FREQ + ORA_MAX_F,     /* number of phase offsets */
  ORA_SE_OFF,                             /* ORA_MAX_P offsets in rad */
  ORA_SE_S = ORA_SE_OFF + ORA_MAX_P,      /* source intensity s */
  ORA_SE_LEN
};
/* screen-space constants and optional output channels */
enum {
  ORA_CO_DIL = 0, ORA_CO_AMAX, ORA_CO_AMIN, ORA_CO_TMIN, ORA_CO_GUARD,
  ORA_CO_SIGMA, ORA_CO_TW, ORA_CO_TH,
  ORA_CO_PHASOR, /* != 0: add the Eq. 3 phasor (Re, Im per frequency) */
  ORA_CO_DEPTH,  /* != 0: add the Eq. 5 mean depth (one-way T)         */
  ORA_CO_NSH,    /* 0: scalar reflectivity; 1, 4, 9, 16: SH of degree
                    0..3, r = max(0, 0.5 + sum_l sh_l Y_l(dir)), dir the
                    unit vector from the optical centre to the Gaussian */
  ORA_CO_LEN
};
/* ambiguity margins (relative): a lower-precision implementation may take
 * a decision the other way when the oracle's value is this close to it */
enum { ORA_EPS_ALPHA = 0, ORA_EPS_T, ORA_EPS_Z, ORA_EPS_RECT, ORA_EPS_LEN };
/* per (frame, Gaussian) projected record ("splat") */
enum {
  ORA_SP_VIS = 0, ORA_SP_U, ORA_SP_V, ORA_SP_CA, ORA_SP_CB, ORA_SP_CC,
  ORA_SP_OPA, ORA_SP_Z, ORA_SP_D, ORA_SP_RAD,
  ORA_SP_X0, ORA_SP_Y0, ORA_SP_X1, ORA_SP_Y1,     /* nominal tile rect */
  ORA_SP_MX0, ORA_SP_MY0, ORA_SP_MX1, ORA_SP_MY1, /* outer (may-cover) rect */
  ORA_SP_IX0, ORA_SP_IY0, ORA_SP_IX1, ORA_SP_IY1, /* inner (surely-covers) */
  ORA_SP_UNCERT,  /* 1: the cull decision itself is within margin */
  ORA_SP_AMP,     /* A = s r / d^2 */
  ORA_SP_FEAT,    /* A sin psi_f, A cos psi_f (f = 0..F-1), then A */
  ORA_SP_LEN = ORA_SP_FEAT + ORA_MAX_FEAT
};
/* per-pixel ambiguity flags */
enum {
  ORA_AMB_ALPHA_MIN = 1, /* an alpha within margin of the skip threshold */
  ORA_AMB_TMIN = 2,      /* the early-stop test within margin of T_min */
  ORA_AMB_ORDER = 4,     /* two contributing Gaussians with near-equal depth */
  ORA_AMB_CLAMP = 8,     /* o G within margin of the alpha clamp (grad only) */
  ORA_AMB_RECT = 16,     /* a contributing Gaussian whose tile membership or
                            cull decision is within margin of flipping */
  ORA_AMB_POWER = 32     /* exponent within margin of the power > 0 skip */
};

#ifdef __cplusplus
extern "C" {
#endif

int ora_splat_len(void);
int ora_num_threads(void);
/* OpenMP threads of the following calls (n > 0; for timing). */
void ora_set_threads(int n);

/* Project all n Gaussians for one frame (Sec. 3; 3DGS EWA convention).
 * params: means[n*3], coeffs[n*9] (c1 xyz, c2 xyz, c3 xyz), scales[n*3],
 * quats[n*4] (w,x,y,z, any norm), opacity[n], amplitude[n], delta[n*3] or
 * NULL, sh[n*ORA_MAX_SH] (read when consts[ORA_CO_NSH] > 0) or NULL.
 * eps[ORA_EPS_LEN] sets the margins behind ORA_SP_UNCERT and the outer/inner
 * rects.  out: splats[n * ORA_SP_LEN]. */
void ora_project(int n, const double* means, const double* coeffs,
                 const double* scales, const double* quats,
                 const double* opacity, const double* amplitude,
                 const double* delta, const double* sh, const double* frame,
                 const double* sensor, const double* consts,
                 const double* eps, double* splats);

/* Real spherical harmonic basis function l (0..15, degree-major) at the unit
 * vector (x, y, z). */
double ora_sh_basis(int l, double x, double y, double z);

/* Raw C-ToF samples for a list of pixels of one frame (Eq. 4).
 * pix[npix*2] = (x, y) pixel indices; bg[C]; out[npix*C]; tfinal[npix];
 * ambig[npix] (ORA_AMB_* flags); ncontrib[npix] (# composited Gaussians).
 * Channels: the F*P raw samples (frequency-major), the ambient channel, then
 * with ORA_CO_PHASOR the phasor Re, Im of each frequency (Eq. 3:
 * p = p_bg T_N + sum 2 A_k exp(i psi_k) alpha_k T_k^2), then with
 * ORA_CO_DEPTH the mean depth sum d_k alpha_k T_k (Eq. 5, one-way T, no
 * background term). */
void ora_render_pixels(int n, const double* splats, const double* frame,
                       const double* sensor, const double* consts,
                       const double* bg, const double* eps, int npix,
                       const int32_t* pix, double* out, double* tfinal,
                       int32_t* ambig, int32_t* ncontrib);

/* Instrumentation of one pixel (x, y): the composited Gaussians' alpha_k and
 * transmittance T_k before them (one-way), front to back, up to max_steps of
 * them; *tfinal = T_N.  Returns the number composited. */
int ora_pixel_steps(int n, const double* splats, const double* sensor,
                    const double* consts, const double* eps, int x, int y,
                    int max_steps, double* alpha, double* trans, double* tfinal);

/* Full frame: out[C*H*W] (channel-major), tfinal[H*W], ambig[H*W],
 * ncontrib[H*W]. */
void ora_render_frame(int n, const double* splats, const double* frame,
                      const double* sensor, const double* consts,
                      const double* bg, const double* eps, double* out,
                      double* tfinal, int32_t* ambig, int32_t* ncontrib);

/* Whole tiles of one frame, and every valid result of their ambiguous
 * pixels.  tiles[ntiles*2] = (tx, ty); pixels are taken tile by tile,
 * row-major, inside the image: pix[npix*2] = (x, y), out[npix*C] (samples as
 * in ora_render_pixels), tfinal[npix], ambig[npix].  For every pixel with a
 * value-changing ambiguity flag, the walk is re-run with its near-threshold
 * decisions (alpha floor, power > 0 skip, T_min stop, near-equal depth order,
 * uncertain tile membership) taken the other way -- up to three at once,
 * each re-run's own near-threshold decisions included, at most max_alt walks
 * per pixel, the first the nominal one -- and each walk's samples go to
 * alt_out[i*C] with alt_pix[i] = its pixel's index, for i < alt_cap.
 * *n_alt = walks produced (may exceed alt_cap: then the rest are dropped);
 * *n_capped = pixels whose search stopped at max_alt.  Returns npix. */
int64_t ora_render_tiles(int n, const double* splats, const double* frame,
                         const double* sensor, const double* consts, const double* bg,
                         const double* eps, int ntiles, const int32_t* tiles, double* out,
                         double* tfinal, int32_t* ambig, int32_t* pix, int max_alt,
                         int64_t alt_cap, double* alt_out, int64_t* alt_pix,
                         int64_t* n_alt, int64_t* n_capped);
/* Gradient of L = sum dout * out for one frame w.r.t. the per-Gaussian 2D
 * record (u, v, conic a, b, c, opacity, features[2F+1], distance d) -- the
 * Eq. S3 recursion for the squared-transmittance channels and the 3DGS
 * one-way recursion for the mean depth.  dout[C*H*W]; pixels whose dout is
 * all zero are skipped.  g2d[n * (7 + 2F+1)] is ACCUMULATED into; dbg[C]
 * accumulated (may be NULL). */
void ora_backward_2d(int n, const double* splats, const double* frame,
                     const double* sensor, const double* consts,
                     const double* bg, const double* dout, double* g2d,
                     double* dbg);

/* Chain the 2D-record gradient of one frame to the Gaussian parameters
 * through the projection with its exact complex-step Jacobian.
 * grads[n * ORA_NPARAM] ACCUMULATED (mu3 c9 s3 q4 o r delta3 sh16). */
void ora_backward_params(int n, const double* means, const double* coeffs,
                         const double* scales, const double* quats,
                         const double* opacity, const double* amplitude,
                         const double* delta, const double* sh, const double* frame,
                         const double* sensor, const double* consts,
                         const double* splats, const double* g2d,
                         double* grads);

/* Bit-exact binning contract (integer work, decided in FP32 like a
 * single-precision implementation must).  For frame b and Gaussian g with
 * radius[b*n+g] > 0 the tile rectangle is
 *   [floor((u-r)/TW), floor((u+r)/TW)+1) x [floor((v-r)/TH), floor((v+r)/TH)+1)
 * clamped to the tile grid, each operation in single precision.  Each covered
 * tile emits key = ((b*tiles + tile) << 32) | bits(z), value = g; the pairs
 * are ordered by (key, value).  ranges[(b*tiles+tile)*2 + {0,1}] = [start,
 * end); an empty tile gets [k, k) with k the count of instances in the tiles
 * before it.  Returns the instance count, or -1 if it exceeds capacity. */
int64_t ora_bin_f32(int n, int frames, const float* u, const float* v,
                    const int32_t* radius, const float* z, int width,
                    int height, int tile_w, int tile_h, int64_t capacity,
                    uint64_t* keys, uint32_t* values, uint32_t* ranges);

#ifdef __cplusplus
}
#endif
#endif
