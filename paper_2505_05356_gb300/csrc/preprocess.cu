// preprocess.cu -- deformation, EWA projection and C-ToF features per
// (frame, Gaussian), and the backward chain rule back to the Gaussian
// parameters (summed over frames in-thread, so the sum order is fixed).
//
// Forward per (frame b, Gaussian g), Sec. 3 and the 3DGS projection it uses:
//   x   = mu + c1 t + c2 t^2 + c3 t^3 + delta_b            (deformation)
//         (under Eq. 7 each t^k is replaced by its linear interpolation
//         between the frame's two timesteps; the table holds the weights)
//   p   = R x + t_cam; cull if p_z <= near
//   d   = |x - o| = distance to the optical centre o = -R^T t_cam (equal to
//         |p| for an orthonormal R; taken from o so that a rounded R does
//         not perturb it)
//   Sigma = Rq diag(s)^2 Rq^T,  Rq from the normalised quaternion
//   J   = [[fx/z, 0, -fx tx/z], [0, fy/z, -fy ty/z]], tx, ty = p_x/z, p_y/z
//         clamped to +-guard * half fov
//   cov = (J R) Sigma (J R)^T + dilation I; cull if det <= 0
//   conic = cov^-1, radius = ceil(sigma_cut sqrt(lambda_max)) (discriminant
//   floored at 0.1), (u, v) = (fx p_x/z + cx, fy p_y/z + cy)
//   A = s r / d^2; features A sin psi_f, A cos psi_f (psi_f = 4 pi d f / c),
//   and A for the ambient channel.  r is the scalar amplitude, or (Sec. 3,
//   view-dependent reflectivity) max(0, 0.5 + sum_l sh_l Y_l(w)) with w the
//   world-space unit vector from the optical centre, w = (x - o) / d.
// The record keeps the conic scaled by -log2(e)/2 (and -log2(e) for the
// cross term) and log2 of the opacity, so that compositing evaluates
// o exp(power) as one ex2; 1/o follows the features.
#include "gftorf_internal.cuh"

namespace gftorf {
namespace {

constexpr double kLog2e = 1.4426950408889634074;
constexpr double kPiD = 3.14159265358979323846;

template <typename Real>
__device__ __forceinline__ Real rsqrt_t(Real x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

// Real spherical harmonics of degree 0..3 (orthonormal on the unit sphere,
// no Condon-Shortley phase), ordered by degree, then m = -l..l.  Constants:
//   Y0 = 1/(2 sqrt(pi)), K1 = sqrt(3/(4 pi)),
//   K2a = sqrt(15/pi)/2, K2b = sqrt(5/pi)/4, K2c = sqrt(15/pi)/4,
//   K3a = sqrt(35/(2 pi))/4, K3b = sqrt(105/pi)/2, K3c = sqrt(21/(2 pi))/4,
//   K3d = sqrt(7/pi)/4, K3e = sqrt(105/pi)/4.
constexpr double kY0 = 0.28209479177387814, kK1 = 0.4886025119029199,
                 kK2a = 1.0925484305920792, kK2b = 0.31539156525252005,
                 kK2c = 0.5462742152960396, kK3a = 0.5900435899266435,
                 kK3b = 2.890611442640554, kK3c = 0.4570457994644658,
                 kK3d = 0.3731763325901154, kK3e = 1.445305721320277;

template <typename Real>
__device__ __forceinline__ void sh_basis(Real x, Real y, Real z, Real* Y) {
  const Real xx = x * x, yy = y * y, zz = z * z;
  Y[0] = Real(kY0);
  Y[1] = Real(kK1) * y;
  Y[2] = Real(kK1) * z;
  Y[3] = Real(kK1) * x;
  Y[4] = Real(kK2a) * x * y;
  Y[5] = Real(kK2a) * y * z;
  Y[6] = Real(kK2b) * (Real(2) * zz - xx - yy);
  Y[7] = Real(kK2a) * x * z;
  Y[8] = Real(kK2c) * (xx - yy);
  Y[9] = Real(kK3a) * y * (Real(3) * xx - yy);
  Y[10] = Real(kK3b) * x * y * z;
  Y[11] = Real(kK3c) * y * (Real(4) * zz - xx - yy);
  Y[12] = Real(kK3d) * z * (Real(2) * zz - Real(3) * xx - Real(3) * yy);
  Y[13] = Real(kK3c) * x * (Real(4) * zz - xx - yy);
  Y[14] = Real(kK3e) * z * (xx - yy);
  Y[15] = Real(kK3a) * x * (xx - Real(3) * yy);
}

// g = sum_l c_l grad Y_l at (x, y, z), the basis taken as polynomials on R^3
template <typename Real>
__device__ __forceinline__ void sh_grad(const Real* c, Real x, Real y, Real z, Real* g) {
  const Real xx = x * x, yy = y * y, zz = z * z;
  const Real K1 = Real(kK1), K2a = Real(kK2a), K2b = Real(kK2b), K2c = Real(kK2c);
  const Real K3a = Real(kK3a), K3b = Real(kK3b), K3c = Real(kK3c), K3d = Real(kK3d),
             K3e = Real(kK3e);
  Real gx = K1 * c[3], gy = K1 * c[1], gz = K1 * c[2];
  gx += K2a * (c[4] * y + c[7] * z) - Real(2) * K2b * c[6] * x + Real(2) * K2c * c[8] * x;
  gy += K2a * (c[4] * x + c[5] * z) - Real(2) * K2b * c[6] * y - Real(2) * K2c * c[8] * y;
  gz += K2a * (c[5] * y + c[7] * x) + Real(4) * K2b * c[6] * z;
  // degree 3
  gx += c[9] * K3a * Real(6) * x * y + c[10] * K3b * y * z - c[11] * K3c * Real(2) * x * y -
        c[12] * K3d * Real(6) * x * z + c[13] * K3c * (Real(4) * zz - Real(3) * xx - yy) +
        c[14] * K3e * Real(2) * x * z + c[15] * K3a * Real(3) * (xx - yy);
  gy += c[9] * K3a * Real(3) * (xx - yy) + c[10] * K3b * x * z +
        c[11] * K3c * (Real(4) * zz - xx - Real(3) * yy) - c[12] * K3d * Real(6) * y * z -
        c[13] * K3c * Real(2) * x * y - c[14] * K3e * Real(2) * y * z -
        c[15] * K3a * Real(6) * x * y;
  gz += c[10] * K3b * x * y + c[11] * K3c * Real(8) * y * z +
        c[12] * K3d * (Real(6) * zz - Real(3) * xx - Real(3) * yy) +
        c[13] * K3c * Real(8) * x * z + c[14] * K3e * (xx - yy);
  g[0] = gx, g[1] = gy, g[2] = gz;
}

// sum_c R[c] x[c] + t, compensated: each product's rounding error is exact
// (fma(a, b, -ab)) and each sum's by Knuth's two-sum, and the collected error
// is added once at the end, so the result is within about one rounding of the
// exact value.  A general rigid camera then moves a footprint centre no more
// than the identity camera does (where p = x is exact).
// (every step with its own rounding: the compiler must not contract them)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename Real>
__device__ __forceinline__ Real dot3_plus(const Real* R, const Real* x, Real t) {
  Real s = t, err = Real(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Real pr = mul_rn(R[c], x[c]);
    const Real pe = fma_rn(R[c], x[c], -pr);
    const Real sn = add_rn(s, pr);
    const Real bb = sub_rn(sn, s);
    const Real se = add_rn(sub_rn(s, sub_rn(sn, bb)), sub_rn(pr, bb));
    s = sn;
    err = add_rn(err, add_rn(pe, se));
  }
  return add_rn(s, err);
}

template <typename Real>
struct Params {
  Real mu[3], c[9], s[3], q[4], o, amp;
  bool has_c;
};

// SH coefficients of Gaussian g, zero beyond n_sh
template <typename Real>
__device__ __forceinline__ void load_sh(const gftorf_gaussians& G, int g, int nsh, Real* c) {
  const Real* src = static_cast<const Real*>(G.sh) + (size_t)nsh * g;
#pragma unroll
  for (int l = 0; l < kMaxSh; ++l) c[l] = l < nsh ? src[l] : Real(0);
}

// r = max(0, 0.5 + sum_l c_l Y_l(w)), w = e / d with e = x - o (world frame);
// returns the unclamped value in *val and w in w[3]
template <typename Real>
__device__ __forceinline__ Real sh_reflectivity(const Real* c, const Real* e, Real d, Real* w,
                                                Real* val) {
  const Real id = Real(1) / d;
#pragma unroll
  for (int a = 0; a < 3; ++a) w[a] = e[a] * id;
  Real Y[kMaxSh];
  sh_basis<Real>(w[0], w[1], w[2], Y);
  Real v = Real(0.5);
#pragma unroll
  for (int l = 0; l < kMaxSh; ++l) v += c[l] * Y[l];
  *val = v;
  return v > Real(0) ? v : Real(0);
}

template <typename Real>
__device__ __forceinline__ void load_params(const gftorf_gaussians& G, int g,
                                            Params<Real>& P) {
  const Real* mu = static_cast<const Real*>(G.means) + 3 * (size_t)g;
  const Real* sc = static_cast<const Real*>(G.scales) + 3 * (size_t)g;
  const Real* qq = static_cast<const Real*>(G.quats) + 4 * (size_t)g;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    P.mu[a] = mu[a];
    P.s[a] = sc[a];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) P.q[a] = qq[a];
  P.has_c = G.coeffs != nullptr;
  if (P.has_c) {
    const Real* cc = static_cast<const Real*>(G.coeffs) + 9 * (size_t)g;
#pragma unroll
    for (int a = 0; a < 9; ++a) P.c[a] = cc[a];
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a) P.c[a] = Real(0);
  }
  P.o = static_cast<const Real*>(G.opacity)[g];
  P.amp = G.amplitude ? static_cast<const Real*>(G.amplitude)[g] : Real(0);
}

// Forward geometry shared by the forward kernel and the backward recompute.
template <typename Real>
struct Geo {
  Real x[3], p[3];
  Real e[3];  // x - o
  Real iz, d;
  Real qn[4], inv_qlen;  // normalised quaternion and 1/|q|
  Real Rq[9], M[9], S[6];  // S: Sigma (00, 01, 02, 11, 12, 22)
  Real tx, ty;
  bool clx, cly;
  Real Tm[6];
  Real cov[3];  // 00, 01, 11 (dilated)
  Real det;
};

template <typename Real>
__device__ __forceinline__ void geometry(const Params<Real>& P,
                                         const FrameT<Real>& fr, const Real* delta,
                                         Real dil, Geo<Real>& Q) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Real x = P.mu[a] + (P.c[a] * fr.tp[0] + P.c[3 + a] * fr.tp[1] + P.c[6 + a] * fr.tp[2]);
    if (delta) x += delta[a];
    Q.x[a] = x;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const Real Rr[3] = {(Real)fr.R[3 * r], (Real)fr.R[3 * r + 1], (Real)fr.R[3 * r + 2]};
    Q.p[r] = dot3_plus<Real>(Rr, Q.x, (Real)fr.t[r]);
  }
  Q.iz = Real(1) / Q.p[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) Q.e[a] = Q.x[a] - (Real)fr.o[a];
  Q.d = sqrt(Q.e[0] * Q.e[0] + Q.e[1] * Q.e[1] + Q.e[2] * Q.e[2]);

  Real ql2 = P.q[0] * P.q[0] + P.q[1] * P.q[1] + P.q[2] * P.q[2] + P.q[3] * P.q[3];
  Q.inv_qlen = rsqrt_t<Real>(ql2);
  const Real w = P.q[0] * Q.inv_qlen, x = P.q[1] * Q.inv_qlen,
             y = P.q[2] * Q.inv_qlen, z = P.q[3] * Q.inv_qlen;
  Q.qn[0] = w, Q.qn[1] = x, Q.qn[2] = y, Q.qn[3] = z;
  Q.Rq[0] = 1 - 2 * (y * y + z * z);
  Q.Rq[1] = 2 * (x * y - w * z);
  Q.Rq[2] = 2 * (x * z + w * y);
  Q.Rq[3] = 2 * (x * y + w * z);
  Q.Rq[4] = 1 - 2 * (x * x + z * z);
  Q.Rq[5] = 2 * (y * z - w * x);
  Q.Rq[6] = 2 * (x * z - w * y);
  Q.Rq[7] = 2 * (y * z + w * x);
  Q.Rq[8] = 1 - 2 * (x * x + y * y);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q.M[3 * i + j] = Q.Rq[3 * i + j] * P.s[j];
  // Sigma = M M^T
  auto dot3 = [&](int i, int j) {
    return Q.M[3 * i] * Q.M[3 * j] + Q.M[3 * i + 1] * Q.M[3 * j + 1] +
           Q.M[3 * i + 2] * Q.M[3 * j + 2];
  };
  Q.S[0] = dot3(0, 0);
  Q.S[1] = dot3(0, 1);
  Q.S[2] = dot3(0, 2);
  Q.S[3] = dot3(1, 1);
  Q.S[4] = dot3(1, 2);
  Q.S[5] = dot3(2, 2);

  const Real fx = (Real)fr.fx, fy = (Real)fr.fy;
  const Real limx = (Real)fr.limx, limy = (Real)fr.limy;
  Real tx = Q.p[0] * Q.iz, ty = Q.p[1] * Q.iz;
  Q.clx = !(tx >= -limx && tx <= limx);
  Q.cly = !(ty >= -limy && ty <= limy);
  tx = fmin(limx, fmax(-limx, tx));
  ty = fmin(limy, fmax(-limy, ty));
  Q.tx = tx, Q.ty = ty;
  const Real J00 = fx * Q.iz, J02 = -fx * tx * Q.iz;
  const Real J11 = fy * Q.iz, J12 = -fy * ty * Q.iz;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    Q.Tm[j] = J00 * (Real)fr.R[j] + J02 * (Real)fr.R[6 + j];
    Q.Tm[3 + j] = J11 * (Real)fr.R[3 + j] + J12 * (Real)fr.R[6 + j];
  }
  // cov = Tm S Tm^T
  Real TS[6];  // Tm * Sigma (2x3)
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const Real* a = Q.Tm + 3 * i;
    TS[3 * i + 0] = a[0] * Q.S[0] + a[1] * Q.S[1] + a[2] * Q.S[2];
    TS[3 * i + 1] = a[0] * Q.S[1] + a[1] * Q.S[3] + a[2] * Q.S[4];
    TS[3 * i + 2] = a[0] * Q.S[2] + a[1] * Q.S[4] + a[2] * Q.S[5];
  }
  Q.cov[0] = TS[0] * Q.Tm[0] + TS[1] * Q.Tm[1] + TS[2] * Q.Tm[2] + dil;
  Q.cov[1] = TS[0] * Q.Tm[3] + TS[1] * Q.Tm[4] + TS[2] * Q.Tm[5];
  Q.cov[2] = TS[3] * Q.Tm[3] + TS[4] * Q.Tm[4] + TS[5] * Q.Tm[5] + dil;
  Q.det = Q.cov[0] * Q.cov[2] - Q.cov[1] * Q.cov[1];
}

template <typename Real, int F, bool SH>
__global__ void __launch_bounds__(256)
    preprocess_kernel(gftorf_gaussians G, const TableT<Real>* __restrict__ tab,
                      Header* __restrict__ hdr, Real* __restrict__ rec,
                      uint2* __restrict__ rect, uint32_t* __restrict__ zkey,
                      int N, int TW, int TH, int tiles_x, int tiles_y,
                      int rec_stride, int cull, int nsh) {
  constexpr int NF = 2 * F + 1;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  bool visible = false;
  if (g < N) {
    const FrameT<Real>& fr = tab->fr[b];
    Params<Real> P;
    load_params<Real>(G, g, P);
    const Real* delta =
        G.delta ? static_cast<const Real*>(G.delta) + ((size_t)b * N + g) * 3 : nullptr;
    Geo<Real> Q;
    geometry<Real>(P, fr, delta, (Real)tab->dilation, Q);
    const size_t bg = (size_t)b * N + g;
    uint2 rr = make_uint2(0, 0);
    uint32_t key = kCulledKey;
    if (Q.p[2] > (Real)fr.near_plane && Q.det > Real(0)) {
      const Real inv_det = Real(1) / Q.det;
      const Real ca = Q.cov[2] * inv_det, cb = -Q.cov[1] * inv_det,
                 cc = Q.cov[0] * inv_det;
      const Real mid = Real(0.5) * (Q.cov[0] + Q.cov[2]);
      const Real lam = mid + sqrt(fmax(Real(0.1), mid * mid - Q.det));
      const Real rad = ceil((Real)tab->sigma_cut * sqrt(lam));
      const int r = rad < Real(1 << 20) ? (int)rad : (1 << 20);
      const Real u = (Real)fr.fx * Q.p[0] * Q.iz + (Real)fr.cx;
      const Real v = (Real)fr.fy * Q.p[1] * Q.iz + (Real)fr.cy;
      int x0, y0, x1, y1;
      tile_rect((float)u, (float)v, r, TW, TH, tiles_x, tiles_y, x0, y0, x1, y1);
      if (cull) {
        // alpha = o G >= alpha_min only inside the ellipse
        // delta^T cov^-1 delta <= kappa = 2 ln(o / alpha_min); its bounding box
        // (plus slack for rounding) bounds every tile a pixel of which can
        // composite this Gaussian
        const Real kappa = Real(2) * log(P.o / (Real)tab->alpha_min);
        if (!(kappa >= Real(0))) {
          x1 = x0;  // never reaches alpha_min
        } else {
          const float ex = (float)(sqrt(kappa * Q.cov[0]) * Real(1.001) + Real(0.5));
          const float ey = (float)(sqrt(kappa * Q.cov[2]) * Real(1.001) + Real(0.5));
          tile_rect_xy((float)u, (float)v, fminf((float)r, ex), fminf((float)r, ey), TW, TH,
                       tiles_x, tiles_y, x0, y0, x1, y1);
        }
      }
      if (x0 < x1 && y0 < y1) {
        visible = true;
        rr = pack_rect(x0, y0, x1, y1);
        key = __float_as_uint((float)Q.p[2]);
        // assemble the record in registers, store it as 16-byte vectors
        constexpr int RSC = (8 + NF + 16 / sizeof(Real) - 1) / (16 / sizeof(Real)) *
                            (16 / sizeof(Real));
        Real o[RSC];
        o[0] = u;
        o[1] = v;
        o[2] = Real(-0.5 * kLog2e) * ca;
        o[3] = Real(-kLog2e) * cb;
        o[4] = Real(-0.5 * kLog2e) * cc;
        o[5] = log2(P.o);  // alpha = 2^(power2 + log2 o)
        Real refl = P.amp;
        if (SH) {
          Real c[kMaxSh], w[3], val;
          load_sh<Real>(G, g, nsh, c);
          refl = sh_reflectivity<Real>(c, Q.e, Q.d, w, &val);
        }
        const Real A = tab->source * refl / (Q.d * Q.d);
#pragma unroll
        for (int f = 0; f < F; ++f) {
          Real sn, cs;
          sincospi_t(tab->kf[f] * Q.d, &sn, &cs);
          o[6 + 2 * f] = A * sn;
          o[7 + 2 * f] = A * cs;
        }
        o[6 + 2 * F] = A;
        o[6 + NF] = Real(1) / P.o;  // recovers G = alpha / o in the backward
        o[7 + NF] = Q.d;            // d_k of the mean depth (Eq. 5)
#pragma unroll
        for (int k = 8 + NF; k < RSC; ++k) o[k] = Real(0);
        float4* dst = reinterpret_cast<float4*>(rec + bg * RSC);
        const float4* srcv = reinterpret_cast<const float4*>(o);
#pragma unroll
        for (int k = 0; k < RSC * (int)sizeof(Real) / 16; ++k) dst[k] = srcv[k];
      }
    }
    rect[bg] = rr;
    zkey[bg] = key;
  }
  // visible count per frame, one atomic per warp
  const unsigned m = __ballot_sync(0xffffffffu, visible);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(&hdr->vis[b], (uint32_t)__popc(m));
}

// ---------------------------------------------------------------------------
// backward: d(record) of every frame -> d(parameters); frames looped in-thread
// ---------------------------------------------------------------------------
// 4 CTAs (16 warps) per SM for the scalar-reflectivity float kernels (<= 128
// registers); the SH variants carry 32 more live values and run at 3; the
// double-precision (checking) variants are left unconstrained
template <typename Real, int F, bool SH>
__global__ void __launch_bounds__(128, sizeof(Real) == 8 ? 1 : (SH ? 3 : 4))
    preprocess_bwd_kernel(gftorf_gaussians G, gftorf_gradients D,
                          const TableT<Real>* __restrict__ tab,
                          const uint2* __restrict__ rect,
                          const Real* __restrict__ g2d, int g2d_stride, int N,
                          int B, int nsh) {
  constexpr int NF = 2 * F + 1;
  constexpr int NS = SH ? kMaxSh : 1;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  Params<Real> P;
  load_params<Real>(G, g, P);
  Real csh[NS], gsh[NS];
#pragma unroll
  for (int l = 0; l < NS; ++l) gsh[l] = Real(0);
  if (SH) load_sh<Real>(G, g, nsh, csh);
  Real gmu[3] = {0, 0, 0}, gc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  Real gs[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, go = 0, gamp = 0;
  const Real dil = (Real)tab->dilation;
  // frame b + 1's rectangle and 2D-gradient row (7 + NF values, the row
  // stride) are loaded while frame b is processed; they are used only where
  // the rectangle says visible, as before
  constexpr int RW = 7 + NF;
  uint2 rr_next = rect[g];
  Real row_next[RW];
#pragma unroll
  for (int i = 0; i < RW; ++i) row_next[i] = g2d[(size_t)g * g2d_stride + i];
  for (int b = 0; b < B; ++b) {
    const size_t bg = (size_t)b * N + g;
    Real* gdelta = D.delta ? static_cast<Real*>(D.delta) + bg * 3 : nullptr;
    const uint2 rr = rr_next;
    Real row[RW];
#pragma unroll
    for (int i = 0; i < RW; ++i) row[i] = row_next[i];
    if (b + 1 < B) {
      const size_t bn = bg + (size_t)N;
      rr_next = rect[bn];
#pragma unroll
      for (int i = 0; i < RW; ++i) row_next[i] = g2d[bn * g2d_stride + i];
    }
    Real gu = 0, gv = 0, ga = 0, gb = 0, gcn = 0, gop = 0, gdist = 0, gf[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) gf[f] = 0;
    bool any = false;
    if (rr.x != rr.y || rr.x != 0) {  // visible in this frame
      gu = row[0], gv = row[1], ga = row[2], gb = row[3], gcn = row[4], gop = row[5];
      gdist = row[6 + NF];  // through the mean depth's d_k
      any = gu != 0 || gv != 0 || ga != 0 || gb != 0 || gcn != 0 || gop != 0 || gdist != 0;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        gf[f] = row[6 + f];
        any |= gf[f] != 0;
      }
    }
    if (!any) {
      if (gdelta) gdelta[0] = gdelta[1] = gdelta[2] = Real(0);
      continue;
    }
    const FrameT<Real>& fr = tab->fr[b];
    const Real* delta =
        G.delta ? static_cast<const Real*>(G.delta) + bg * 3 : nullptr;
    Geo<Real> Q;
    geometry<Real>(P, fr, delta, dil, Q);
    const Real fx = (Real)fr.fx, fy = (Real)fr.fy;
    const Real iz = Q.iz, iz2 = iz * iz;

    // --- C-ToF features: A = s r / d^2, psi_f = pi kf d ---
    const Real id = Real(1) / Q.d;
    Real refl = P.amp, wv[3] = {0, 0, 0}, val = 0;
    if (SH) refl = sh_reflectivity<Real>(csh, Q.e, Q.d, wv, &val);
    const Real A = (Real)tab->source * refl * id * id;
    Real gA = gf[2 * F];
    Real gd = 0;
#pragma unroll
    for (int f = 0; f < F; ++f) {
      Real s, c;
      const Real kf = (Real)tab->kf[f];
      sincospi_t(kf * Q.d, &s, &c);
      gA += gf[2 * f] * s + gf[2 * f + 1] * c;
      const Real gpsi = A * (gf[2 * f] * c - gf[2 * f + 1] * s);
      gd += gpsi * Real(kPiD) * kf;
    }
    const Real gr_ = gA * (Real)tab->source * id * id;  // dL/dr
    Real gw[3] = {0, 0, 0};  // dL/d(x - o) through the SH direction
    if (!SH) {
      gamp += gr_;
    } else if (val > Real(0)) {
      Real Y[kMaxSh];
      sh_basis<Real>(wv[0], wv[1], wv[2], Y);
#pragma unroll
      for (int l = 0; l < NS; ++l) gsh[l] += gr_ * Y[l];
      // w = v / |v|: dL/dv = (I - w w^T) dL/dw / |v|
      Real gdir[3];
      sh_grad<Real>(csh, wv[0], wv[1], wv[2], gdir);
      const Real wd = wv[0] * gdir[0] + wv[1] * gdir[1] + wv[2] * gdir[2];
#pragma unroll
      for (int a = 0; a < 3; ++a) gw[a] = gr_ * (gdir[a] - wv[a] * wd) * id;
    }
    gd += gA * Real(-2) * A * id + gdist;
    // d = |x - o|: dL/dx += gd (x - o) / d, in world coordinates
#pragma unroll
    for (int a = 0; a < 3; ++a) gw[a] += gd * Q.e[a] * id;
    Real gp[3] = {0, 0, 0};

    // --- mean 2D ---
    gp[0] += gu * fx * iz;
    gp[1] += gv * fy * iz;
    gp[2] -= (gu * fx * Q.p[0] + gv * fy * Q.p[1]) * iz2;

    // --- conic = cov^-1: dL/dcov = -C Gm C, Gm = [[ga, gb/2], [gb/2, gc]] ---
    const Real inv_det = Real(1) / Q.det;
    const Real ca = Q.cov[2] * inv_det, cb = -Q.cov[1] * inv_det, cc = Q.cov[0] * inv_det;
    const Real hb = Real(0.5) * gb;
    // X = C Gm
    const Real X00 = ca * ga + cb * hb, X01 = ca * hb + cb * gcn;
    const Real X10 = cb * ga + cc * hb, X11 = cb * hb + cc * gcn;
    const Real K00 = -(X00 * ca + X01 * cb);
    const Real K01 = -(X00 * cb + X01 * cc);
    const Real K11 = -(X10 * cb + X11 * cc);
    // symmetric gradient of cov as a matrix: [[K00, K01], [K01, K11]]
    // --- cov = Tm S Tm^T (+dil): dS = Tm^T K Tm, dTm = 2 K Tm S ---
    Real KT[6];  // K Tm (2x3)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      KT[j] = K00 * Q.Tm[j] + K01 * Q.Tm[3 + j];
      KT[3 + j] = K01 * Q.Tm[j] + K11 * Q.Tm[3 + j];
    }
    Real dS[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) dS[3 * i + j] = Q.Tm[i] * KT[j] + Q.Tm[3 + i] * KT[3 + j];
    const Real Sf[9] = {Q.S[0], Q.S[1], Q.S[2], Q.S[1], Q.S[3], Q.S[4], Q.S[2], Q.S[4], Q.S[5]};
    Real dTm[6];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dTm[3 * i + j] = Real(2) * (KT[3 * i] * Sf[j] + KT[3 * i + 1] * Sf[3 + j] +
                                     KT[3 * i + 2] * Sf[6 + j]);
    // --- Tm = J R ---
    Real dJ00 = 0, dJ02 = 0, dJ11 = 0, dJ12 = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      dJ00 += dTm[j] * (Real)fr.R[j];
      dJ02 += dTm[j] * (Real)fr.R[6 + j];
      dJ11 += dTm[3 + j] * (Real)fr.R[3 + j];
      dJ12 += dTm[3 + j] * (Real)fr.R[6 + j];
    }
    // J00 = fx/z, J02 = -fx tx/z, J11 = fy/z, J12 = -fy ty/z
    Real gz = -dJ00 * fx * iz2 + dJ02 * fx * Q.tx * iz2 - dJ11 * fy * iz2 +
              dJ12 * fy * Q.ty * iz2;
    if (!Q.clx) {
      const Real gtx = -dJ02 * fx * iz;
      gp[0] += gtx * iz;
      gz -= gtx * Q.p[0] * iz2;
    }
    if (!Q.cly) {
      const Real gty = -dJ12 * fy * iz;
      gp[1] += gty * iz;
      gz -= gty * Q.p[1] * iz2;
    }
    gp[2] += gz;
    // --- p = R x + t ---
    Real gx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      gx[a] = (Real)fr.R[a] * gp[0] + (Real)fr.R[3 + a] * gp[1] + (Real)fr.R[6 + a] * gp[2] +
              gw[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      gmu[a] += gx[a];
      gc[a] += gx[a] * fr.tp[0];
      gc[3 + a] += gx[a] * fr.tp[1];
      gc[6 + a] += gx[a] * fr.tp[2];
    }
    if (gdelta) {
      gdelta[0] = gx[0];
      gdelta[1] = gx[1];
      gdelta[2] = gx[2];
    }
    // --- Sigma = M M^T: dM = 2 dS M (dS symmetric) ---
    Real dM[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dM[3 * i + j] = Real(2) * (dS[3 * i] * Q.M[j] + dS[3 * i + 1] * Q.M[3 + j] +
                                   dS[3 * i + 2] * Q.M[6 + j]);
    // --- M = Rq diag(s) ---
    Real dR[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        gs[j] += dM[3 * i + j] * Q.Rq[3 * i + j];
        dR[3 * i + j] = dM[3 * i + j] * P.s[j];
      }
    // --- Rq(qn) ---
    const Real w = Q.qn[0], x = Q.qn[1], y = Q.qn[2], z = Q.qn[3];
    Real dqn[4];
    dqn[0] = 2 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dqn[1] = 2 * (y * dR[1] + z * dR[2] + y * dR[3] - 2 * x * dR[4] - w * dR[5] +
                  z * dR[6] + w * dR[7] - 2 * x * dR[8]);
    dqn[2] = 2 * (-2 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] -
                  w * dR[6] + z * dR[7] - 2 * y * dR[8]);
    dqn[3] = 2 * (-2 * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2 * z * dR[4] +
                  y * dR[5] + x * dR[6] + y * dR[7]);
    // --- qn = q / |q| ---
    const Real dot = w * dqn[0] + x * dqn[1] + y * dqn[2] + z * dqn[3];
#pragma unroll
    for (int a = 0; a < 4; ++a) gq[a] += (dqn[a] - Q.qn[a] * dot) * Q.inv_qlen;
    go += gop;
  }
  if (D.means) {
    Real* o = static_cast<Real*>(D.means) + 3 * (size_t)g;
    o[0] = gmu[0], o[1] = gmu[1], o[2] = gmu[2];
  }
  if (D.coeffs) {
    Real* o = static_cast<Real*>(D.coeffs) + 9 * (size_t)g;
#pragma unroll
    for (int a = 0; a < 9; ++a) o[a] = gc[a];
  }
  if (D.scales) {
    Real* o = static_cast<Real*>(D.scales) + 3 * (size_t)g;
    o[0] = gs[0], o[1] = gs[1], o[2] = gs[2];
  }
  if (D.quats) {
    Real* o = static_cast<Real*>(D.quats) + 4 * (size_t)g;
    o[0] = gq[0], o[1] = gq[1], o[2] = gq[2], o[3] = gq[3];
  }
  if (D.opacity) static_cast<Real*>(D.opacity)[g] = go;
  if (D.amplitude) static_cast<Real*>(D.amplitude)[g] = gamp;
  if (SH && D.sh) {
    Real* o = static_cast<Real*>(D.sh) + (size_t)nsh * g;
#pragma unroll
    for (int l = 0; l < NS; ++l)
      if (l < nsh) o[l] = gsh[l];
  }
}

}  // namespace

template <typename Real>
void launch_preprocess(const Layout& L, const gftorf_gaussians& g,
                       unsigned char* ws, cudaStream_t st) {
  if (L.N == 0) return;
  dim3 grid((L.N + 255) / 256, L.B);
  auto* tab = table_of<Real>(ws, L.off_table);
  auto* hdr = at<Header>(ws, L.off_header);
  auto* rec = at<Real>(ws, L.off_rec);
  auto* rect = at<uint2>(ws, L.off_rect);
  auto* zkey = at<uint32_t>(ws, L.off_zkey);
#define GFTORF_PRE(FF)                                                         \
  if (L.nsh)                                                                   \
    preprocess_kernel<Real, FF, true><<<grid, 256, 0, st>>>(                   \
        g, tab, hdr, rec, rect, zkey, L.N, L.TW, L.TH, L.tiles_x, L.tiles_y,   \
        L.rec_stride, L.cull, L.nsh);                                          \
  else                                                                         \
    preprocess_kernel<Real, FF, false><<<grid, 256, 0, st>>>(                  \
        g, tab, hdr, rec, rect, zkey, L.N, L.TW, L.TH, L.tiles_x, L.tiles_y,   \
        L.rec_stride, L.cull, 0)
  switch (L.F) {
    case 1: GFTORF_PRE(1); break;
    case 2: GFTORF_PRE(2); break;
    case 3: GFTORF_PRE(3); break;
    default: GFTORF_PRE(4); break;
  }
  count_launches(1);
#undef GFTORF_PRE
}

template <typename Real>
void launch_preprocess_bwd(const Layout& L, const gftorf_gaussians& g,
                           const gftorf_gradients& gr, unsigned char* ws,
                           cudaStream_t st) {
  if (L.N == 0) return;
  dim3 grid((L.N + 127) / 128);
  auto* tab = table_of<Real>(ws, L.off_table);
  auto* rect = at<const uint2>(ws, L.off_rect);
  auto* g2d = at<const Real>(ws, L.off_g2d);
#define GFTORF_PREB(FF)                                                        \
  if (L.nsh)                                                                   \
    preprocess_bwd_kernel<Real, FF, true><<<grid, 128, 0, st>>>(               \
        g, gr, tab, rect, g2d, L.g2d_stride, L.N, L.B, L.nsh);                 \
  else                                                                         \
    preprocess_bwd_kernel<Real, FF, false><<<grid, 128, 0, st>>>(              \
        g, gr, tab, rect, g2d, L.g2d_stride, L.N, L.B, 0)
  switch (L.F) {
    case 1: GFTORF_PREB(1); break;
    case 2: GFTORF_PREB(2); break;
    case 3: GFTORF_PREB(3); break;
    default: GFTORF_PREB(4); break;
  }
  count_launches(1);
#undef GFTORF_PREB
}

template void launch_preprocess<float>(const Layout&, const gftorf_gaussians&,
                                       unsigned char*, cudaStream_t);
template void launch_preprocess<double>(const Layout&, const gftorf_gaussians&,
                                        unsigned char*, cudaStream_t);
template void launch_preprocess_bwd<float>(const Layout&, const gftorf_gaussians&,
                                           const gftorf_gradients&,
                                           unsigned char*, cudaStream_t);
template void launch_preprocess_bwd<double>(const Layout&,
                                            const gftorf_gaussians&,
                                            const gftorf_gradients&,
                                            unsigned char*, cudaStream_t);

}  // namespace gftorf
