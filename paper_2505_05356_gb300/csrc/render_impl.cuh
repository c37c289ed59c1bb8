// render_impl.cuh -- per-tile compositing of raw C-ToF samples (Eq. 4) and its
// backward re-walk (Eq. S3).  A thread owns PPT (1, 2 or 4) vertically
// adjacent pixels of a tile, so each staged Gaussian record, its column
// offset and (backward) its warp reduction serve PPT pixels; one CTA per
// (frame, tile part) or persistent CTAs pulling such items from a queue (a
// tile 64 wide is composited in 32x32 parts, one CTA each).
//
// Forward, per pixel, front to back over the tile's depth-ordered list:
//   alpha = min(alpha_max, 2^(power2 + log2 o)), power2 = log2(e) * power
//   skip if power2 > 0 or alpha < alpha_min
//   stop (without compositing) if T (1 - alpha) < t_min
//   w = alpha T^2;  acc_f += w feature_f  (A sin psi_f, A cos psi_f, A)
//   T <- T (1 - alpha)
// Epilogue: Q_fj = cos(phi_j) S_f + sin(phi_j) C_f + bg_fj T,
//           ambient = I + bg_amb T   (sum_k A_k sin(psi_k + phi_j) w_k + bg T)
// Backward, per pixel, back to front from its last composited Gaussian:
//   T_k = T_{k+1} / (1 - alpha_k)   (one-way transmittance recovered)
//   dL/dalpha_k = sum_c g_c T_k^2 (q_kc - 2 (1 - alpha_k) acc_c)
//                 - g_T T_N / (1 - alpha_k)
//   acc_c <- alpha_k q_kc + (1 - alpha_k)^2 acc_c          (Eq. S3)
// with g_c the gradient of the accumulators (the raw samples are linear in
// them) and g_T = sum_c bg_c dL/dQ_c.  Per-Gaussian sums over the CTA's
// pixels: warp shuffle reduction, shared-memory accumulation, then one
// global atomic per value per CTA.
#pragma once

#include "gftorf_internal.cuh"



namespace gftorf {
namespace {

constexpr double kLn2 = 0.69314718055994530942;

// Reals per record: u, v, scaled conic (3), log2 o, 2F+1 features, 1/o,
// distance d, padded to 16 bytes
template <int F>
struct RecStrideF {
  static constexpr int value = ((8 + 2 * F + 1) + 3) / 4 * 4;
};
template <int F>
struct RecStrideD {
  static constexpr int value = ((8 + 2 * F + 1) + 1) / 2 * 2;
};
template <typename Real, int F>
constexpr int rec_stride() {
  return sizeof(Real) == 4 ? RecStrideF<F>::value : RecStrideD<F>::value;
}

// one rounding per operation, so forward and backward evaluate alpha with
// bit-identical results (the backward replays the forward's decisions)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// 1/a: one rcp.approx in single precision (the backward's T recovery and the
// tile test's half-reciprocals tolerate its ~1 ulp), exact in double
__device__ __forceinline__ float rcp_fast(float a) { return rcp_approx(a); }
__device__ __forceinline__ double rcp_fast(double a) { return 1.0 / a; }

template <typename Real>
__device__ __forceinline__ Real warp_sum(Real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduce GS values over the 32 lanes of a warp by recursive halving: at
// each step a lane keeps one half of its values and trades the other half
// with its partner, so the warp spends ceil(GS/2) + ceil(GS/4) + ... shuffles
// instead of 5 GS.  Afterwards lane L holds the full sum of value index
// `slot_of_lane` (computed once per thread by butterfly_slot).
template <int LEN, int OFF>
struct Fold {
  template <typename Real>
  static __device__ __forceinline__ void run(Real* v, int lane) {
    constexpr int H = (LEN + 1) / 2;
    const bool up = (lane & OFF) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const Real lo = v[i];
      const Real hi = (i + H < LEN) ? v[i + H] : Real(0);
      const Real keep = up ? hi : lo;
      const Real send = up ? lo : hi;
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
    }
    Fold<H, OFF / 2>::run(v, lane);
  }
};
template <int LEN>
struct Fold<LEN, 0> {
  template <typename Real>
  static __device__ __forceinline__ void run(Real*, int) {}
};

// value index whose warp total lane `lane` ends with after Fold<GS, 16>;
// -1 for lanes that end with padding only
template <int GS>
__device__ __forceinline__ int butterfly_slot(int lane) {
  int start = 0, end = GS, len = GS;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const int h = (len + 1) / 2;
    if (lane & off) {
      start += h;
    } else {
      end = min(end, start + h);
    }
    len = h;
  }
  return start < end ? start : -1;
}

// One CTA composites a CW x CH part of a binning tile (CW = min(TW, 32); CH =
// 32 for tiles 32 or more wide, else TH): a 64x32 tile (whose list is shared)
// is taken by S = 2 CTAs, a 64x64 one by 4, each testing the records against
// its own part, so each pixel composites the same records in the same order
// as with 32x32 tiles.
struct TileCtx {
  int b, tile, tx, ty;
  int x0, y0;  // first pixel column and row of the CTA's part of the tile
};

struct RenderGeom {
  int N, W, H, TW, TH, tiles_x, NT, P, C, rec_stride, B, cull, phasor;
  int CW, CH, SX, S;  // columns and rows per CTA, CTAs across and per tile
};

__device__ __forceinline__ TileCtx tile_of(uint32_t item, const RenderGeom& rg) {
  TileCtx c;
  const uint32_t per_frame = (uint32_t)rg.NT * rg.S;
  c.b = item / per_frame;
  const uint32_t sub = item - (uint32_t)c.b * per_frame;
  c.tile = sub / rg.S;
  const int part = (int)(sub - (uint32_t)c.tile * rg.S);
  c.ty = c.tile / rg.tiles_x;
  c.tx = c.tile - c.ty * rg.tiles_x;
  const int py = part / rg.SX, pxp = part - py * rg.SX;
  c.x0 = c.tx * rg.TW + pxp * rg.CW;
  c.y0 = c.ty * rg.TH + py * rg.CH;
  return c;
}

// The pixels of a thread and the block of its warp, tile-local.  Tiles at
// most 16 wide: thread t owns column t % TW, rows from (t / TW) PPT, so a warp
// covers 32 / TW whole rows of PPT-pixel strips.  32-wide tiles: warps cover
// 16 x 2 PPT blocks, TW / 16 of them across, so that a warp's pixels stay a
// compact block whatever the tile's width (its record mask tests that block).
struct ThreadPix {
  int lx, ly0;             // first pixel of the thread
  int wx0, wx1, wy0, wy1;  // the warp's block (inclusive)
};
template <int PPT>
__device__ __forceinline__ ThreadPix thread_pixels(int tid, int TW) {
  ThreadPix t;
  const int lane = tid & 31, wid = tid >> 5;
  if (TW <= 16) {
    t.lx = tid % TW;
    t.ly0 = (tid / TW) * PPT;
    t.wx0 = 0;
    t.wx1 = TW - 1;
    t.wy0 = ((wid << 5) / TW) * PPT;
    t.wy1 = (((wid << 5) + 31) / TW) * PPT + PPT - 1;
  } else {
    const int across = TW / 16, bx = wid % across, by = wid / across;
    t.lx = bx * 16 + (lane & 15);
    t.ly0 = by * 2 * PPT + (lane >> 4) * PPT;
    t.wx0 = bx * 16;
    t.wx1 = bx * 16 + 15;
    t.wy0 = by * 2 * PPT;
    t.wy1 = t.wy0 + 2 * PPT - 1;
  }
  return t;
}

// Can the Gaussian of record r reach alpha_min at some pixel centre of the
// tile whose centres span [cx0, cx1] x [cy0, cy1]?  With A, B, C the negated
// scaled conic, alpha >= alpha_min means A dx^2 + B dx dy + C dy^2 <= K,
// K = log2(o / alpha_min); the quadratic's minimum over the rectangle is 0
// if the centre lies inside, else it lies on an edge at the clamped 1-D
// minimiser.  Generous slack keeps the test conservative under rounding.
template <typename Real>
__device__ __forceinline__ bool tile_hit(const Real* r, Real cx0, Real cx1, Real cy0,
                                         Real cy1, Real log2_amin) {
  const Real K = r[5] - log2_amin;
  if (!(K >= Real(-1e-3))) return false;
  const Real lx = cx0 - r[0], hx = cx1 - r[0], ly = cy0 - r[1], hy = cy1 - r[1];
  if (lx <= Real(0) && hx >= Real(0) && ly <= Real(0) && hy >= Real(0)) return true;
  const Real A = -r[2], B = -r[3], C = -r[4];
  const Real hA = Real(0.5) * rcp_fast(A), hC = Real(0.5) * rcp_fast(C);
  Real m = Real(1e30);
  // horizontal edges dy = ly, hy
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const Real dy = e ? hy : ly;
    const Real dx = fmin(hx, fmax(lx, -B * dy * hA));
    m = fmin(m, (A * dx + B * dy) * dx + C * dy * dy);
  }
  // vertical edges dx = lx, hx
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const Real dx = e ? hx : lx;
    const Real dy = fmin(hy, fmax(ly, -B * dx * hC));
    m = fmin(m, (A * dx + B * dy) * dx + C * dy * dy);
  }
  return m <= K * Real(1.001) + Real(1e-3);
}

// Per-warp masks of staged records: at most 512 threads per CTA, so at most
// 16 warps and 16 words of 32 records each.
constexpr int kMaskWords = 16;

// Block-wide stable compaction: returns this thread's slot among the kept
// ones (valid when keep) and the number kept; s_cnt holds >= 32 ints.
__device__ __forceinline__ int block_compact(bool keep, int* s_cnt, int& pos) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, keep);
  if (lane == 0) s_cnt[wid] = __popc(bal);
  __syncthreads();
  int off = 0, total = 0;
  for (int w = 0; w < nw; ++w) {
    const int c = s_cnt[w];
    off += w < wid ? c : 0;
    total += c;
  }
  pos = off + __popc(bal & lanemask_lt());
  return total;
}

// number of entries of the increasing array a[0..n) below x
__device__ __forceinline__ int count_below(const uint32_t* a, int n, uint32_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// forward: thread (lx, row group) owns PPT vertically adjacent pixels
// ---------------------------------------------------------------------------

// log2 of o G for one Gaussian at pixel offset (dx, dy), evaluated as a
// quadratic in dy whose coefficients depend only on the column:
//   cc' dy^2 + (cb' dx) dy + (ca' dx^2 + log2 o),
// cb_dx and a_lo computed once per column and shared by its PPT pixels.  One
// rounding per operation, so the backward replays the forward's decisions
// bit for bit.  power2 > log2 o is the "power > 0" skip of the method.
template <typename Real>
struct Column {
  Real dx, cb_dx, a_lo;
};
template <typename Real>
__device__ __forceinline__ Column<Real> column_of(const Real* r, Real fpx) {
  Column<Real> c;
  c.dx = sub_rn(r[0], fpx);
  c.cb_dx = mul_rn(r[3], c.dx);
  c.a_lo = fma_rn(mul_rn(r[2], c.dx), c.dx, r[5]);
  return c;
}
template <typename Real>
__device__ __forceinline__ Real log2_oG(const Real* r, const Column<Real>& c, Real dy) {
  return fma_rn(fma_rn(r[4], dy, c.cb_dx), dy, c.a_lo);
}

// Two FP32 values in one 64-bit register pair, for the packed FP32x2
// instructions of this architecture: each lane is the IEEE round-to-nearest
// result of the scalar operation, so packed and scalar code agree bit for
// bit, while one instruction issue does the work of two.
struct F2 {
  unsigned long long v;
};
__device__ __forceinline__ F2 pack2(float a, float b) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(F2 x, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ F2 sub2_rn(F2 a, F2 b) {
  F2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 fma2_rn(F2 a, F2 b, F2 c) {
  F2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}

// log2_oG of the PPT pixels of one column: pairs of pixels in packed FP32x2
// (the same roundings as log2_oG); the double instantiation stays scalar
template <int PPT>
__device__ __forceinline__ void log2_oG_column(const float* r, const Column<float>& c,
                                               const float* fpy, float* lg) {
  if constexpr (PPT % 2 == 0) {
    const F2 r1 = pack2(r[1], r[1]), r4 = pack2(r[4], r[4]);
    const F2 cb = pack2(c.cb_dx, c.cb_dx), alo = pack2(c.a_lo, c.a_lo);
#pragma unroll
    for (int h = 0; h < PPT / 2; ++h) {
      const F2 dy = sub2_rn(r1, pack2(fpy[2 * h], fpy[2 * h + 1]));
      unpack2(fma2_rn(fma2_rn(r4, dy, cb), dy, alo), lg[2 * h], lg[2 * h + 1]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < PPT; ++k) lg[k] = log2_oG(r, c, sub_rn(r[1], fpy[k]));
  }
}
template <int PPT>
__device__ __forceinline__ void log2_oG_column(const double* r, const Column<double>& c,
                                               const double* fpy, double* lg) {
#pragma unroll
  for (int k = 0; k < PPT; ++k) lg[k] = log2_oG(r, c, sub_rn(r[1], fpy[k]));
}

// Resident CTAs per SM the compiler is asked to fit (register budget).  Only
// the 4-pixel variants are register limited: with 128 threads (16x32 tile) the
// forward keeps 7 CTAs (<= 72 registers), the backward 6 (<= 80); with 256
// threads (32x32 tile, WIDE) 3 of either (<= 85).
template <int PPT, bool BWD, bool WIDE>
struct kMinBlocks {
  static constexpr int value = WIDE ? 3 : (PPT == 4 ? (BWD ? 6 : 7) : 0);
};
template <int PPT, bool WIDE>
struct kMaxThreads {
  static constexpr int value = (WIDE ? 1024 : 512) / PPT;
};

template <typename Real, int F, int PPT, bool DEPTH, bool COUNT>
__device__ __forceinline__ void render_tile_fwd(
    const TileCtx& tc, const RenderGeom& rg, const TableT<Real>* __restrict__ tab,
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ values,
    const Real* __restrict__ rec, const Real* __restrict__ bg,
    Real* __restrict__ out, Real* __restrict__ tfinal,
    uint32_t* __restrict__ nlast, Real* s_rec, Real* s_stage, uint32_t* s_idx,
    int* s_cnt, unsigned* s_mask, Header* __restrict__ hdr) {
  constexpr int NF = 2 * F + 1;
  constexpr int RS = rec_stride<Real, F>();
  constexpr unsigned ALL = (1u << PPT) - 1u;
  const int nthr = blockDim.x, tid = threadIdx.x;
  const ThreadPix tp = thread_pixels<PPT>(tid, rg.CW);
  const int lx = tp.lx, ly0 = tp.ly0;
  const int px = tc.x0 + lx, py0 = tc.y0 + ly0;
  const Real fpx = (Real)px + Real(0.5);
  Real fpy[PPT];
  unsigned done = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    fpy[k] = (Real)(py0 + k) + Real(0.5);
    if (!(px < rg.W && py0 + k < rg.H)) done |= 1u << k;
  }
  const unsigned outside = done;
  const Real amax = (Real)tab->alpha_max, amin = (Real)tab->alpha_min;
  const Real tmin = (Real)tab->t_min;
  const uint2 range = ranges[(size_t)tc.b * rg.NT + tc.tile];
  const Real* frec = rec + (size_t)tc.b * rg.N * RS;

  Real T[PPT], acc[PPT][NF], accD[PPT];  // accD: mean depth (DEPTH only)
  uint32_t last[PPT];
  uint32_t evals = 0;  // evaluated pairs (COUNT only)
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    T[k] = 1;
    accD[k] = 0;
    last[k] = range.x;
#pragma unroll
    for (int f = 0; f < NF; ++f) acc[k][f] = 0;
  }

  constexpr int V4 = RS * (int)sizeof(Real) / 16;
  const Real cx0 = (Real)tc.x0 + Real(0.5), cx1 = cx0 + (Real)(rg.CW - 1);
  const Real cy0 = (Real)tc.y0 + Real(0.5), cy1 = cy0 + (Real)(rg.CH - 1);
  const Real log2_amin = log2(amin);
  // this warp's block of the tile (pixel centres)
  const int lane = tid & 31, wid = tid >> 5;
  const Real wx0 = cx0 + (Real)tp.wx0, wx1 = cx0 + (Real)tp.wx1;
  const Real wy0 = cy0 + (Real)tp.wy0, wy1 = cy0 + (Real)tp.wy1;
  uint32_t wevals = 0;  // pairs of records that reach the warp's rows (COUNT only)
  for (uint32_t base = range.x; base < range.y; base += nthr) {
    if (__syncthreads_count(done == ALL) == nthr) break;
    // stage the batch, then keep only the records that can reach alpha_min
    // in this tile, compacted in list order
    const uint32_t i = base + tid;
    bool keep = false;
    if (i < range.y) {
      const float4* src = reinterpret_cast<const float4*>(frec + (size_t)values[i] * RS);
      float4* stg = reinterpret_cast<float4*>(s_stage + tid * RS);
#pragma unroll
      for (int k = 0; k < V4; ++k) stg[k] = __ldg(src + k);
      keep = !rg.cull || tile_hit<Real>(s_stage + tid * RS, cx0, cx1, cy0, cy1, log2_amin);
    }
    int pos;
    const int cnt = block_compact(keep, s_cnt, pos);
    if (keep) {
      const float4* stg = reinterpret_cast<const float4*>(s_stage + tid * RS);
      float4* dst = reinterpret_cast<float4*>(s_rec + pos * RS);
#pragma unroll
      for (int k = 0; k < V4; ++k) dst[k] = stg[k];
      s_idx[pos] = i;
    }
    __syncthreads();
    // records that can reach alpha_min at a pixel centre of this warp's block
    // (the tile test on the warp's rectangle): bit j of word q is record
    // 32 q + j; the others are skipped by every pixel of the warp
    const int nq = (cnt + 31) >> 5;
    for (int q = 0; q < nq; ++q) {
      const int j = (q << 5) + lane;
      const bool hit = j < cnt && (!rg.cull || tile_hit<Real>(s_rec + j * RS, wx0, wx1, wy0, wy1,
                                                               log2_amin));
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) s_mask[wid * kMaskWords + q] = m;
    }
    __syncwarp();
    for (int q = 0; q < nq && done != ALL; ++q) {
      unsigned m = s_mask[wid * kMaskWords + q];
      // the pair-counting instantiation walks every record (its count is the
      // tile lists' candidate pairs) and counts the warp's records apart
      unsigned walk = COUNT ? (q + 1 < nq || (cnt & 31) == 0 ? 0xffffffffu
                                                             : (1u << (cnt & 31)) - 1u)
                            : m;
      while (walk && done != ALL) {
        const int bit = __ffs(walk) - 1;
        walk &= walk - 1;
        const int j = (q << 5) + bit;
        const Real* r = s_rec + j * RS;
        const Column<Real> col = column_of(r, fpx);
        // the exponents of all PPT pixels first (independent chains), then
        // each pixel's decisions
        Real lg[PPT], oG[PPT];
        log2_oG_column<PPT>(r, col, fpy, lg);
#pragma unroll
        for (int k = 0; k < PPT; ++k) oG[k] = ex2_approx(lg[k]);
        const uint32_t jn = s_idx[j] + 1;  // list entries up to this one
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (done & (1u << k)) continue;
          if (COUNT) {
            ++evals;
            wevals += (m >> bit) & 1u;
          }
          const Real alpha = oG[k] < amax ? oG[k] : amax;
          if (lg[k] > r[5] || alpha < amin) continue;
          const Real aT = alpha * T[k];
          const Real tn = T[k] - aT;  // T (1 - alpha)
          if (tn < tmin) {
            done |= 1u << k;
            continue;
          }
          const Real w = aT * T[k];
#pragma unroll
          for (int f = 0; f < NF; ++f) acc[k][f] += w * r[6 + f];
          if (DEPTH) accD[k] += aT * r[7 + NF];  // Eq. 5: one-way T
          T[k] = tn;
          last[k] = jn;
        }
      }
    }
  }
  if (COUNT) {
    unsigned long long e = evals, ew = wevals;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      ew += __shfl_xor_sync(0xffffffffu, ew, o);
    }
    if ((tid & 31) == 0 && e) atomicAdd(&hdr->pairs, e);
    if ((tid & 31) == 0 && ew) atomicAdd(&hdr->pairs_warp, ew);
  }
  const size_t HW = (size_t)rg.W * rg.H;
  const Real* bgb = bg + (size_t)tc.b * rg.C;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    if (outside & (1u << k)) continue;
    const size_t pix = (size_t)(py0 + k) * rg.W + px;
    Real* o = out + (size_t)tc.b * rg.C * HW + pix;
    for (int f = 0; f < F; ++f)
      for (int j = 0; j < rg.P; ++j)
        o[(size_t)(f * rg.P + j) * HW] = (Real)tab->fr[tc.b].cos_off[j] * acc[k][2 * f] +
                                         (Real)tab->fr[tc.b].sin_off[j] * acc[k][2 * f + 1] +
                                         bgb[f * rg.P + j] * T[k];
    o[(size_t)(F * rg.P) * HW] = acc[k][2 * F] + bgb[F * rg.P] * T[k];
    int c = F * rg.P + 1;
    if (rg.phasor) {  // Eq. 3: p = 2 (C_f + i S_f) + p_bg T_N
      for (int f = 0; f < F; ++f, c += 2) {
        o[(size_t)c * HW] = Real(2) * acc[k][2 * f + 1] + bgb[c] * T[k];
        o[(size_t)(c + 1) * HW] = Real(2) * acc[k][2 * f] + bgb[c + 1] * T[k];
      }
    }
    if (DEPTH) o[(size_t)c * HW] = accD[k];
    tfinal[(size_t)tc.b * HW + pix] = T[k];
    nlast[(size_t)tc.b * HW + pix] = last[k] - range.x;
  }
}

template <typename Real, int F, int PPT, bool DEPTH, bool COUNT, bool WIDE>
__global__ void __launch_bounds__(kMaxThreads<PPT, WIDE>::value,
                                  kMinBlocks<PPT, false, WIDE>::value)
    render_fwd_kernel(RenderGeom rg, const TableT<Real>* __restrict__ tab,
                      Header* __restrict__ hdr,
                      const uint2* __restrict__ ranges,
                      const uint32_t* __restrict__ values,
                      const Real* __restrict__ rec, const Real* __restrict__ bg,
                      Real* __restrict__ out, Real* __restrict__ tfinal,
                      uint32_t* __restrict__ nlast, int persistent) {
  constexpr int RS = rec_stride<Real, F>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* s_rec = reinterpret_cast<Real*>(smem_raw);
  Real* s_stage = s_rec + (size_t)blockDim.x * RS;
  uint32_t* s_idx = reinterpret_cast<uint32_t*>(s_stage + (size_t)blockDim.x * RS);
  __shared__ int s_cnt[32];
  __shared__ unsigned s_mask[kMaskWords * kMaskWords];  // [warp][word]
  const uint32_t items = (uint32_t)rg.B * rg.NT * rg.S;
  if (!persistent) {
    const uint32_t item = blockIdx.y * rg.NT * rg.S + blockIdx.x;
    render_tile_fwd<Real, F, PPT, DEPTH, COUNT>(tile_of(item, rg), rg, tab, ranges,
                                         values, rec, bg, out, tfinal, nlast, s_rec, s_stage,
                                         s_idx, s_cnt, s_mask, hdr);
    return;
  }
  __shared__ uint32_t s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&hdr->queue[0], 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= items) break;
    render_tile_fwd<Real, F, PPT, DEPTH, COUNT>(tile_of(item, rg), rg, tab, ranges,
                                         values, rec, bg, out, tfinal, nlast, s_rec, s_stage,
                                         s_idx, s_cnt, s_mask, hdr);
  }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
template <typename Real, int F, int PPT, bool DEPTH>
__device__ __forceinline__ void render_tile_bwd(
    const TileCtx& tc, const RenderGeom& rg, const TableT<Real>* __restrict__ tab,
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ values,
    const Real* __restrict__ rec, const Real* __restrict__ bg,
    const Real* __restrict__ dout, const Real* __restrict__ tfinal,
    const uint32_t* __restrict__ nlast, Real* __restrict__ g2d, int g2d_stride,
    Real* __restrict__ dbg, Real* s_rec, Real* s_grad, uint32_t* s_id,
    Real* s_red, uint32_t* s_idx, int* s_cnt, Real* s_stage, unsigned* s_mask) {
  constexpr int NF = 2 * F + 1;
  constexpr int GS = 6 + NF + (DEPTH ? 1 : 0);
  constexpr int RS = rec_stride<Real, F>();
  const int nthr = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nwarps = nthr >> 5;
  const ThreadPix tp = thread_pixels<PPT>(tid, rg.CW);
  const int lx = tp.lx, ly0 = tp.ly0;
  const int px = tc.x0 + lx, py0 = tc.y0 + ly0;
  const Real fpx = (Real)px + Real(0.5);
  const Real amax = (Real)tab->alpha_max, amin = (Real)tab->alpha_min;
  const uint2 range = ranges[(size_t)tc.b * rg.NT + tc.tile];
  const Real* frec = rec + (size_t)tc.b * rg.N * RS;
  const size_t HW = (size_t)rg.W * rg.H;
  const Real* bgb = bg + (size_t)tc.b * rg.C;

  // fold dL/dQ into accumulator gradients, per pixel
  Real fpy[PPT], Tf[PPT], gTf[PPT], gacc[PPT][NF], gD[PPT];
  int nl[PPT];
  bool inside[PPT];
  int thread_n = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    fpy[k] = (Real)(py0 + k) + Real(0.5);
    inside[k] = px < rg.W && py0 + k < rg.H;
#pragma unroll
    for (int f = 0; f < NF; ++f) gacc[k][f] = 0;
    gD[k] = 0;
    Real gT = 0;
    Tf[k] = 1;
    nl[k] = 0;
    if (inside[k]) {
      const size_t pix = (size_t)(py0 + k) * rg.W + px;
      const Real* go = dout + (size_t)tc.b * rg.C * HW + pix;
      Tf[k] = tfinal[(size_t)tc.b * HW + pix];
      nl[k] = (int)nlast[(size_t)tc.b * HW + pix];
      for (int f = 0; f < F; ++f)
        for (int j = 0; j < rg.P; ++j) {
          const Real gq = go[(size_t)(f * rg.P + j) * HW];
          gacc[k][2 * f] += (Real)tab->fr[tc.b].cos_off[j] * gq;
          gacc[k][2 * f + 1] += (Real)tab->fr[tc.b].sin_off[j] * gq;
          gT += bgb[f * rg.P + j] * gq;
        }
      gacc[k][2 * F] = go[(size_t)(F * rg.P) * HW];
      gT += bgb[F * rg.P] * gacc[k][2 * F];
      int c = F * rg.P + 1;
      if (rg.phasor) {  // Re = 2 C_f, Im = 2 S_f
        for (int f = 0; f < F; ++f, c += 2) {
          const Real gre = go[(size_t)c * HW], gim = go[(size_t)(c + 1) * HW];
          gacc[k][2 * f + 1] += Real(2) * gre;
          gacc[k][2 * f] += Real(2) * gim;
          gT += bgb[c] * gre + bgb[c + 1] * gim;
        }
      }
      if (DEPTH) gD[k] = go[(size_t)c * HW];
    }
    gTf[k] = gT * Tf[k];
    thread_n = max(thread_n, nl[k]);
  }
  // dL/dbg_c = sum over pixels of T_N dL/dQ_c (block reduce, one atomic each)
  if (dbg) {
    for (int c = 0; c < rg.C - (DEPTH ? 1 : 0); ++c) {  // Eq. 5 has no background
      Real v = 0;
#pragma unroll
      for (int k = 0; k < PPT; ++k)
        if (inside[k])
          v += Tf[k] * dout[((size_t)tc.b * rg.C + c) * HW + (size_t)(py0 + k) * rg.W + px];
      v = warp_sum(v);
      if (lane == 0) s_red[wid] = v;
      __syncthreads();
      if (tid == 0) {
        Real s = 0;
        for (int w = 0; w < nwarps; ++w) s += s_red[w];
        if (s != Real(0)) atomicAdd(&dbg[(size_t)tc.b * rg.C + c], s);
      }
      __syncthreads();
    }
  }
  // longest list any pixel of the tile needs
  int maxn = thread_n;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxn = max(maxn, __shfl_xor_sync(0xffffffffu, maxn, o));
  if (lane == 0) reinterpret_cast<int*>(s_red)[wid] = maxn;
  __syncthreads();
  maxn = 0;
  for (int w = 0; w < nwarps; ++w) maxn = max(maxn, reinterpret_cast<int*>(s_red)[w]);
  __syncthreads();

  // Per pixel only the projection of the Eq. S3 accumulators on the pixel's
  // (fixed) accumulator gradient is needed: A = sum_f g_f acc_f obeys the same
  // recursion, A <- alpha (g . q) + (1 - alpha)^2 A.
  // BD likewise projects the one-way mean-depth recursion (DEPTH only):
  // BD <- alpha gD d + (1 - alpha) BD, d depth / d alpha_k = T_k (d_k - accD_k)
  Real T[PPT], A[PPT], BD[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    T[k] = Tf[k];
    A[k] = 0;
    BD[k] = 0;
  }
  const int red_slot = butterfly_slot<GS>(lane);
  const Real ln2 = Real(kLn2);
  Real* gbase = g2d + (size_t)tc.b * rg.N * g2d_stride;

  constexpr int V4 = RS * (int)sizeof(Real) / 16;
  const Real cx0 = (Real)tc.x0 + Real(0.5), cx1 = cx0 + (Real)(rg.CW - 1);
  const Real cy0 = (Real)tc.y0 + Real(0.5), cy1 = cy0 + (Real)(rg.CH - 1);
  const Real log2_amin = log2(amin);
  // this warp's block of the tile (pixel centres)
  const Real wx0 = cx0 + (Real)tp.wx0, wx1 = cx0 + (Real)tp.wx1;
  const Real wy0 = cy0 + (Real)tp.wy0, wy1 = cy0 + (Real)tp.wy1;
  for (int hi = maxn; hi > 0; hi -= nthr) {
    const int lo = max(0, hi - nthr);
    const int cnt = hi - lo;
    // stage entries [lo, hi), keeping the records that can reach alpha_min
    // in this tile (the same test as the forward's, so the same entries)
    bool keep = false;
    uint32_t g = 0;
    if (tid < cnt) {
      g = values[range.x + lo + tid];
      const float4* src = reinterpret_cast<const float4*>(frec + (size_t)g * RS);
      float4* stg = reinterpret_cast<float4*>(s_stage + tid * RS);
#pragma unroll
      for (int k = 0; k < V4; ++k) stg[k] = __ldg(src + k);
      keep = !rg.cull || tile_hit<Real>(s_stage + tid * RS, cx0, cx1, cy0, cy1, log2_amin);
    }
    int pos;
    const int nk = block_compact(keep, s_cnt, pos);
    if (keep) {
      const float4* stg = reinterpret_cast<const float4*>(s_stage + tid * RS);
      float4* dst = reinterpret_cast<float4*>(s_rec + pos * RS);
#pragma unroll
      for (int k = 0; k < V4; ++k) dst[k] = stg[k];
      s_id[pos] = g;
      s_idx[pos] = (uint32_t)(lo + tid);
    }
    for (int k = tid; k < nk * GS; k += nthr) s_grad[k] = Real(0);
    __syncthreads();
    // staged entries [0, my_hi[k]) precede pixel k's last composited one;
    // warps whose pixels all stop before the batch skip it
    int my_hi[PPT];
    int thread_hi = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      my_hi[k] = count_below(s_idx, nk, (uint32_t)nl[k]);
      thread_hi = max(thread_hi, my_hi[k]);
    }
    int warp_hi = thread_hi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) warp_hi = max(warp_hi, __shfl_xor_sync(0xffffffffu, warp_hi, o));
    // records below warp_hi that can reach alpha_min in this warp's block (the
    // forward's warp test, so the same records): bit j of word q is 32 q + j
    const int nq = (warp_hi + 31) >> 5;
    for (int q = 0; q < nq; ++q) {
      const int j = (q << 5) + lane;
      const bool hit = j < warp_hi && (!rg.cull || tile_hit<Real>(s_rec + j * RS, wx0, wx1, wy0,
                                                                   wy1, log2_amin));
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) s_mask[wid * kMaskWords + q] = m;
    }
    __syncwarp();
    for (int q = nq - 1; q >= 0; --q) {
     unsigned m = s_mask[wid * kMaskWords + q];
     while (m) {
      const int bit = 31 - __clz(m);
      m &= ~(1u << bit);
      const int j = (q << 5) + bit;
      const Real* r = s_rec + j * RS;
      Real c[GS];
#pragma unroll
      for (int q = 0; q < GS; ++q) c[q] = 0;
      bool has = false;
      if (j < thread_hi) {
        const Column<Real> col = column_of(r, fpx);
        // moments over this thread's pixels (same column) of dL/dpower:
        // S0 = sum d, S1 = sum d dy, S2 = sum d dy^2 (S0 is also the sum of
        // dL/dalpha o G: where alpha is not clamped, d = dL/dalpha alpha and
        // alpha = o G)
        Real S0 = 0, S1 = 0, S2 = 0;
        Real lgv[PPT];  // exponents of all PPT pixels first (packed pairs)
        log2_oG_column<PPT>(r, col, fpy, lgv);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (j >= my_hi[k]) continue;
          const Real dy = sub_rn(r[1], fpy[k]);
          const Real lg = lgv[k];
          const Real oG = ex2_approx(lg);
          const Real alpha = oG < amax ? oG : amax;
          if (lg > r[5] || alpha < amin) continue;
          has = true;
          const Real oma = Real(1) - alpha;
          const Real rcp = rcp_fast(oma);
          const Real Tk = T[k] * rcp;
          const Real T2 = Tk * Tk;
          Real gq = 0;
#pragma unroll
          for (int f = 0; f < NF; ++f) gq += gacc[k][f] * r[6 + f];
          const Real X = oma * A[k];
          Real dLda = T2 * (gq - Real(2) * X) - gTf[k] * rcp;
          A[k] = alpha * gq + oma * X;
          if (DEPTH) {
            const Real gDd = gD[k] * r[7 + NF];
            dLda += Tk * (gDd - BD[k]);
            c[6 + NF] += gD[k] * alpha * Tk;
            BD[k] = alpha * gDd + oma * BD[k];
          }
          const Real aT2 = alpha * T2;
#pragma unroll
          for (int f = 0; f < NF; ++f) c[6 + f] += gacc[k][f] * aT2;
          T[k] = Tk;
          if (oG < amax) {  // alpha = o G is not clamped: it depends on o, u, v, conic
            const Real d = dLda * alpha;  // d alpha / d power = alpha
            const Real t = d * dy;
            S0 += d;
            S1 += t;
            S2 += t * dy;
          }
        }
        if (has) {
          // moments in dx as well: the gradients of u, v, the conic and o are
          // linear in these sums, so the warp sums them and the flush applies
          // the record's constants once per CTA
          const Real dx = col.dx;
          const Real b = dx * S0;
          c[0] = b;       // sum dx d
          c[1] = dx * b;  // sum dx^2 d
          c[2] = S1;      // sum dy d
          c[3] = dx * S1; // sum dx dy d
          c[4] = S2;      // sum dy^2 d
          c[5] = S0;      // sum dL/dalpha o G
        }
      }
      if (__any_sync(0xffffffffu, has)) {
        Fold<GS, 16>::run(c, lane);
        if (red_slot >= 0 && c[0] != Real(0)) atomicAdd(&s_grad[j * GS + red_slot], c[0]);
      }
     }
    }
    __syncthreads();
    // per record: the 2D gradient from the CTA's sums (alpha = 2^(log2 o +
    // ln2-scaled quadratic), d alpha / d o = alpha / o), one global atomic per
    // non-zero component
    for (int jj = tid; jj < nk; jj += nthr) {
      const Real* rr = s_rec + jj * RS;
      const Real* sg = s_grad + jj * GS;
      Real v[GS];
      v[0] = ln2 * (Real(2) * rr[2] * sg[0] + rr[3] * sg[2]);
      v[1] = ln2 * (Real(2) * rr[4] * sg[2] + rr[3] * sg[0]);
      v[2] = Real(-0.5) * sg[1];
      v[3] = -sg[3];
      v[4] = Real(-0.5) * sg[4];
      v[5] = sg[5] * rr[6 + NF];
#pragma unroll
      for (int q = 6; q < GS; ++q) v[q] = sg[q];
      Real* gr = gbase + (size_t)s_id[jj] * g2d_stride;
#pragma unroll
      for (int q = 0; q < GS; ++q)
        if (v[q] != Real(0)) atomicAdd(&gr[q], v[q]);
    }
    __syncthreads();
  }
}

template <typename Real, int F, int PPT, bool DEPTH, bool WIDE>
__global__ void __launch_bounds__(kMaxThreads<PPT, WIDE>::value,
                                  kMinBlocks<PPT, true, WIDE>::value)
    render_bwd_kernel(RenderGeom rg, const TableT<Real>* __restrict__ tab,
                      Header* __restrict__ hdr,
                      const uint2* __restrict__ ranges,
                      const uint32_t* __restrict__ values,
                      const Real* __restrict__ rec, const Real* __restrict__ bg,
                      const Real* __restrict__ dout,
                      const Real* __restrict__ tfinal,
                      const uint32_t* __restrict__ nlast, Real* __restrict__ g2d,
                      int g2d_stride, Real* __restrict__ dbg, int persistent) {
  constexpr int NF = 2 * F + 1;
  constexpr int GS = 6 + NF + (DEPTH ? 1 : 0);
  constexpr int RS = rec_stride<Real, F>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nthr = blockDim.x;
  Real* s_rec = reinterpret_cast<Real*>(smem_raw);
  Real* s_grad = s_rec + (size_t)nthr * RS;
  Real* s_red = s_grad + (size_t)nthr * GS;
  uint32_t* s_id = reinterpret_cast<uint32_t*>(s_red + 32);
  uint32_t* s_idx = s_id + nthr;
  Real* s_stage = reinterpret_cast<Real*>(s_idx + nthr);
  __shared__ int s_cnt[32];
  __shared__ unsigned s_mask[kMaskWords * kMaskWords];  // [warp][word]
  const uint32_t items = (uint32_t)rg.B * rg.NT * rg.S;
  if (!persistent) {
    const uint32_t item = blockIdx.y * rg.NT * rg.S + blockIdx.x;
    render_tile_bwd<Real, F, PPT, DEPTH>(tile_of(item, rg), rg, tab, ranges,
                                  values, rec, bg, dout, tfinal, nlast, g2d,
                                  g2d_stride, dbg, s_rec, s_grad, s_id, s_red, s_idx, s_cnt,
                                  s_stage, s_mask);
    return;
  }
  __shared__ uint32_t s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&hdr->queue[1], 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= items) break;
    render_tile_bwd<Real, F, PPT, DEPTH>(tile_of(item, rg), rg, tab, ranges,
                                  values, rec, bg, dout, tfinal, nlast, g2d,
                                  g2d_stride, dbg, s_rec, s_grad, s_id, s_red, s_idx, s_cnt,
                                  s_stage, s_mask);
  }
}

RenderGeom geom_of(const Layout& L) {
  RenderGeom g;
  g.N = L.N, g.W = L.W, g.H = L.H, g.TW = L.TW, g.TH = L.TH;
  g.tiles_x = L.tiles_x, g.NT = L.NT, g.P = L.P, g.C = L.C;
  g.rec_stride = L.rec_stride, g.B = L.B, g.cull = L.cull, g.phasor = L.phasor;
  g.CW = L.TW < 32 ? L.TW : 32;
  g.CH = L.TW < 32 ? L.TH : 32;
  g.SX = L.TW / g.CW;
  g.S = g.SX * (L.TH / g.CH);
  return g;
}

template <typename KernelT>
int persistent_grid(KernelT kernel, int threads, size_t smem) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  return sm_count() * (per_sm > 0 ? per_sm : 1);
}

template <typename Real, int F, int PPT, bool DEPTH, bool COUNT, bool WIDE>
void fwd_launch(const Layout& L, const Real* bg, Real* out, unsigned char* ws,
                cudaStream_t st) {
  constexpr int RS = rec_stride<Real, F>();
  const RenderGeom rg = geom_of(L);
  const int threads = rg.CW * rg.CH / PPT;
  const size_t smem = (size_t)threads * (2 * RS * sizeof(Real) + sizeof(uint32_t));
  auto kernel = render_fwd_kernel<Real, F, PPT, DEPTH, COUNT, WIDE>;
  static PerDeviceOnce attr;
  attr.run([&] {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                96 * 1024) == cudaSuccess;
  });
  auto* hdr = at<Header>(ws, L.off_header);
  dim3 grid(L.NT * rg.S, L.B);
  if (L.mode == 1) {
    const int n = persistent_grid(kernel, threads, smem);
    grid = dim3(min(n, L.B * L.NT * rg.S), 1);
    cudaMemsetAsync(&hdr->queue[0], 0, sizeof(uint32_t), st);
  }
  kernel<<<grid, threads, smem, st>>>(
      rg, table_of<Real>(ws, L.off_table), hdr,
      at<const uint2>(ws, L.off_ranges), at<const uint32_t>(ws, L.off_values),
      at<const Real>(ws, L.off_rec), bg, out, at<Real>(ws, L.off_tfinal),
      at<uint32_t>(ws, L.off_nlast), L.mode == 1);
  count_launches(1);
}

template <typename Real, int F, int PPT, bool DEPTH, bool WIDE>
void bwd_launch(const Layout& L, const Real* bg, const Real* dout, Real* dbg,
                unsigned char* ws, cudaStream_t st) {
  constexpr int NF = 2 * F + 1;
  constexpr int GS = 6 + NF + (DEPTH ? 1 : 0);
  constexpr int RS = rec_stride<Real, F>();
  const RenderGeom rg = geom_of(L);
  const int threads = rg.CW * rg.CH / PPT;
  const size_t smem = (size_t)threads * (2 * RS + GS) * sizeof(Real) +
                      32 * sizeof(Real) + (size_t)threads * 2 * sizeof(uint32_t);
  auto kernel = render_bwd_kernel<Real, F, PPT, DEPTH, WIDE>;
  static PerDeviceOnce attr;
  attr.run([&] {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                96 * 1024) == cudaSuccess;
  });
  auto* hdr = at<Header>(ws, L.off_header);
  dim3 grid(L.NT * rg.S, L.B);
  if (L.mode == 1) {
    const int n = persistent_grid(kernel, threads, smem);
    grid = dim3(min(n, L.B * L.NT * rg.S), 1);
    cudaMemsetAsync(&hdr->queue[1], 0, sizeof(uint32_t), st);
  }
  kernel<<<grid, threads, smem, st>>>(
      rg, table_of<Real>(ws, L.off_table), hdr,
      at<const uint2>(ws, L.off_ranges), at<const uint32_t>(ws, L.off_values),
      at<const Real>(ws, L.off_rec), bg, dout, at<const Real>(ws, L.off_tfinal),
      at<const uint32_t>(ws, L.off_nlast), at<Real>(ws, L.off_g2d),
      L.g2d_stride, dbg, L.mode == 1);
  count_launches(1);
}

template <typename Real, int F, bool DEPTH>
void fwd_dispatch(const Layout& L, const Real* bg, Real* out, unsigned char* ws,
                  cudaStream_t st) {
  // 32-wide tiles come with 4 pixels per thread (256 threads)
  if (L.TW > 16) {
    if (L.count_pairs)
      fwd_launch<Real, F, 4, DEPTH, true, true>(L, bg, out, ws, st);
    else
      fwd_launch<Real, F, 4, DEPTH, false, true>(L, bg, out, ws, st);
    return;
  }
  if (L.count_pairs) {
    switch (L.ppt) {
      case 1: fwd_launch<Real, F, 1, DEPTH, true, false>(L, bg, out, ws, st); break;
      case 4: fwd_launch<Real, F, 4, DEPTH, true, false>(L, bg, out, ws, st); break;
      default: fwd_launch<Real, F, 2, DEPTH, true, false>(L, bg, out, ws, st); break;
    }
    return;
  }
  switch (L.ppt) {
    case 1: fwd_launch<Real, F, 1, DEPTH, false, false>(L, bg, out, ws, st); break;
    case 4: fwd_launch<Real, F, 4, DEPTH, false, false>(L, bg, out, ws, st); break;
    default: fwd_launch<Real, F, 2, DEPTH, false, false>(L, bg, out, ws, st); break;
  }
}

template <typename Real, int F, bool DEPTH>
void bwd_dispatch(const Layout& L, const Real* bg, const Real* dout, Real* dbg,
                  unsigned char* ws, cudaStream_t st) {
  if (L.TW > 16) {
    bwd_launch<Real, F, 4, DEPTH, true>(L, bg, dout, dbg, ws, st);
    return;
  }
  switch (L.ppt) {
    case 1: bwd_launch<Real, F, 1, DEPTH, false>(L, bg, dout, dbg, ws, st); break;
    case 4: bwd_launch<Real, F, 4, DEPTH, false>(L, bg, dout, dbg, ws, st); break;
    default: bwd_launch<Real, F, 2, DEPTH, false>(L, bg, dout, dbg, ws, st); break;
  }
}

}  // namespace

template <typename Real, bool DEPTH>
void launch_render_fwd_t(const Layout& L, const Real* bg, Real* out,
                       unsigned char* ws, cudaStream_t st) {
  switch (L.F) {
    case 1: fwd_dispatch<Real, 1, DEPTH>(L, bg, out, ws, st); break;
    case 2: fwd_dispatch<Real, 2, DEPTH>(L, bg, out, ws, st); break;
    case 3: fwd_dispatch<Real, 3, DEPTH>(L, bg, out, ws, st); break;
    default: fwd_dispatch<Real, 4, DEPTH>(L, bg, out, ws, st); break;
  }
}

template <typename Real, bool DEPTH>
void launch_render_bwd_t(const Layout& L, const Real* bg, const Real* dout,
                       Real* dbg, unsigned char* ws, cudaStream_t st) {
  switch (L.F) {
    case 1: bwd_dispatch<Real, 1, DEPTH>(L, bg, dout, dbg, ws, st); break;
    case 2: bwd_dispatch<Real, 2, DEPTH>(L, bg, dout, dbg, ws, st); break;
    case 3: bwd_dispatch<Real, 3, DEPTH>(L, bg, dout, dbg, ws, st); break;
    default: bwd_dispatch<Real, 4, DEPTH>(L, bg, dout, dbg, ws, st); break;
  }
}

}  // namespace gftorf
