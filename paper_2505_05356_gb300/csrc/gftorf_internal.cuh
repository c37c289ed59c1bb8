// gftorf_internal.cuh -- device-side layout and helpers shared by the CUDA
// translation units of libgftorf (sm_103a).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/gftorf.h"

#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>

namespace gftorf {

// ---------------------------------------------------------------------------
// per-device host state: function attributes and device properties belong to
// a device's context, so a process driving several GPUs keeps one copy each
// ---------------------------------------------------------------------------
constexpr int kMaxDevices = 64;

inline int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
  return d;
}

// Runs f() once per device (the current one); returns f's result on the
// call that ran it and the cached result afterwards.  Devices beyond the
// table run f() on every call.
struct PerDeviceOnce {
  std::once_flag flag[kMaxDevices];
  bool ok[kMaxDevices] = {};
  template <typename F>
  bool run(F&& f) {
    const int d = current_device();
    if (d < 0) return f();
    std::call_once(flag[d], [&] { ok[d] = f(); });
    return ok[d];
  }
};

// multiprocessor count of the current device, looked up once per device
inline int sm_count() {
  static std::atomic<int> cache[kMaxDevices];
  const int d = current_device();
  if (d >= 0) {
    const int c = cache[d].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d < 0 ? 0 : d) != cudaSuccess ||
      n <= 0)
    n = 1;
  if (d >= 0) cache[d].store(n, std::memory_order_relaxed);
  return n;
}

// NVTX range over one C-ABI call (a no-op unless a profiler is attached):
// the stages show up by name in timeline tools.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

constexpr int kMaxF = GFTORF_MAX_FREQ;
constexpr int kMaxP = GFTORF_MAX_OFFSETS;
constexpr int kMaxFrames = GFTORF_MAX_FRAMES;
constexpr int kMaxSh = GFTORF_MAX_SH;
constexpr uint32_t kCulledKey = 0xFFFFFFFFu;

// Depth sort geometry: 256 threads, 8 keys each, one tile of 2048 keys.
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
// Tile binning: a chunk of kChunk consecutive instances (in emission order:
// frame, depth rank, tile of the rectangle) per CTA.
constexpr int kChunk = 8192;
// Device-wide scan: elements per CTA (few enough CTAs that they all fit on
// the GPU at once, so the look-back chains stay short) and threads per CTA.
constexpr int kScanTile = 16384;
constexpr int kScanThreads = 512;

// Per-frame camera in device memory.
template <typename T>
struct FrameT {
  T fx, fy, cx, cy;
  T R[9];
  T t[3];
  T near_plane, time;
  T limx, limy;  // guard * half field of view (tan), x and y
  T o[3];        // optical centre -R^T t (world), exact for a non-orthonormal R
  T tp[3];       // deformation weights of c1, c2, c3: (t, t^2, t^3), or their
                 // Eq. 7 interpolation between the frame's two timesteps
  T cos_off[kMaxP], sin_off[kMaxP];  // phase offsets + the frame's own offset
};

// Everything a batch needs besides the arrays: written into the workspace by
// gftorf_preprocess, read by the later kernels.  Kept in double and, for the
// single-precision kernels, in float (conversions from double are slow on
// this part, so FP32 kernels never touch the double copy).
template <typename T>
struct TableT {
  FrameT<T> fr[kMaxFrames];
  T kf[kMaxF];  // 4 f / c: psi / pi per metre of distance
  T source;
  T dilation, alpha_max, alpha_min, t_min, sigma_cut;
};
using Table = TableT<double>;

// Device-side status block at the start of the workspace.
struct Header {
  int32_t status;
  int32_t pad0;
  int64_t count;           // tile instances of the batch
  unsigned long long pairs;  // evaluated (pixel, Gaussian) pairs (when counted)
  unsigned long long pairs_warp;  // of those, the ones in records that reach the
                                  // warp's rows (the rest are skipped per warp)
  uint32_t queue[4];       // persistent work-queue heads (fwd, bwd)
  uint32_t vis[kMaxFrames];  // visible Gaussians per frame
  uint32_t fstart[kMaxFrames + 1];  // first instance of each frame
  uint32_t coff[kMaxFrames + 1];    // first binning chunk of each frame
};

// Host-computed byte layout of the workspace for one gftorf_dims.
struct Layout {
  int B, N, W, H, TW, TH, F, P, C, NF, dtype, real_size, mode;
  int ppt;   // pixels per compositing thread (1, 2 or 4)
  int cull;  // drop (Gaussian, tile) pairs that cannot reach alpha_min
  int count_pairs;  // count evaluated (pixel, Gaussian) pairs in the forward
  int phasor, depth;  // extra output channels (Eq. 3 phasor, Eq. 5 depth)
  int nsh;            // SH reflectivity coefficients per Gaussian (0: scalar)
  int tiles_x, tiles_y, NT;
  int rec_stride;  // Reals per projected record (16-byte multiple)
  int g2d_stride;  // Reals per 2D-gradient row
  int n_dblk;      // depth-sort tiles per frame
  int n_chunk;     // binning chunks of the batch (upper bound)
  int n_scan;      // CTAs of the emission-offset scan
  int scatter_warps;
  int64_t cap;
  size_t off_header, off_table, off_rec, off_rect, off_srect, off_zkey, off_zkey2,
      off_ids, off_ids2, off_dhist, off_dtot, off_ecnt, off_bsum, off_tcnt, off_toff,
      off_ranges,
      off_values, off_tfinal, off_nlast, off_g2d, total;
};

// Host-side count of kernels enqueued by the library (gftorf_kernel_launches).
void count_launches(int n);
int64_t launches_so_far();

// Launch entry points implemented in the .cu files (all on `st`).
template <typename Real>
void launch_preprocess(const Layout& L, const gftorf_gaussians& g,
                       unsigned char* ws, cudaStream_t st);
template <typename Real>
void launch_preprocess_bwd(const Layout& L, const gftorf_gaussians& g,
                           const gftorf_gradients& gr, unsigned char* ws,
                           cudaStream_t st);
void launch_footprints(const Layout& L, const float* u, const float* v,
                       const int32_t* radius, const float* z,
                       unsigned char* ws, cudaStream_t st);
void launch_binning(const Layout& L, unsigned char* ws, cudaStream_t st);
size_t lb_bytes(const Layout& L);  // depth-sort look-back region
void launch_export_keys(const Layout& L, uint64_t* keys, unsigned char* ws,
                        cudaStream_t st);
template <typename Real, bool DEPTH>
void launch_render_fwd_t(const Layout& L, const Real* bg, Real* out,
                         unsigned char* ws, cudaStream_t st);
template <typename Real, bool DEPTH>
void launch_render_bwd_t(const Layout& L, const Real* bg, const Real* dout,
                         Real* dbg, unsigned char* ws, cudaStream_t st);
template <typename Real>
inline void launch_render_fwd(const Layout& L, const Real* bg, Real* out,
                              unsigned char* ws, cudaStream_t st) {
  if (L.depth)
    launch_render_fwd_t<Real, true>(L, bg, out, ws, st);
  else
    launch_render_fwd_t<Real, false>(L, bg, out, ws, st);
}
template <typename Real>
inline void launch_render_bwd(const Layout& L, const Real* bg, const Real* dout,
                              Real* dbg, unsigned char* ws, cudaStream_t st) {
  if (L.depth)
    launch_render_bwd_t<Real, true>(L, bg, dout, dbg, ws, st);
  else
    launch_render_bwd_t<Real, false>(L, bg, dout, dbg, ws, st);
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

template <typename T>
__host__ __device__ inline T* at(unsigned char* ws, size_t off) {
  return reinterpret_cast<T*>(ws + off);
}

// the batch table in the kernels' own precision (the float copy follows the
// double one in the workspace)
template <typename Real>
__host__ __device__ inline const TableT<Real>* table_of(unsigned char* ws, size_t off) {
  return sizeof(Real) == 8 ? reinterpret_cast<const TableT<Real>*>(ws + off)
                           : reinterpret_cast<const TableT<Real>*>(ws + off + sizeof(Table));
}

__device__ __forceinline__ void set_status(Header* h, int32_t code) {
  atomicCAS(&h->status, 0, code);
}

// 2^x with the hardware approximation (PTX ex2.approx.ftz.f32); used on the
// compositing hot path with the conic pre-scaled by log2(e).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double ex2_approx(double x) { return exp2(x); }
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Tile rectangle [x0,x1) x [y0,y1) of the disc of radius r around (u, v),
// every step in single precision with one rounding each (the binning
// contract); clamps are done in float so NaN and huge values are safe.
__device__ __forceinline__ int clamp_tile(float v, int hi) {
  if (!(v > 0.0f)) return 0;
  if (v > (float)hi) return hi;
  return (int)v;
}
__device__ __forceinline__ void tile_rect(float u, float v, int r, int tw,
                                          int th, int tiles_x, int tiles_y,
                                          int& x0, int& y0, int& x1, int& y1) {
  const float rf = (float)r, twf = (float)tw, thf = (float)th;
  x0 = clamp_tile(floorf(__fdiv_rn(__fsub_rn(u, rf), twf)), tiles_x);
  x1 = clamp_tile(__fadd_rn(floorf(__fdiv_rn(__fadd_rn(u, rf), twf)), 1.0f), tiles_x);
  y0 = clamp_tile(floorf(__fdiv_rn(__fsub_rn(v, rf), thf)), tiles_y);
  y1 = clamp_tile(__fadd_rn(floorf(__fdiv_rn(__fadd_rn(v, rf), thf)), 1.0f), tiles_y);
}

// Same rectangle for separate half-widths in x and y (float), used for the
// alpha-ellipse bounding box; it lies inside tile_rect's for rx, ry <= r.
__device__ __forceinline__ void tile_rect_xy(float u, float v, float rx, float ry,
                                             int tw, int th, int tiles_x,
                                             int tiles_y, int& x0, int& y0,
                                             int& x1, int& y1) {
  const float twf = (float)tw, thf = (float)th;
  x0 = clamp_tile(floorf(__fdiv_rn(__fsub_rn(u, rx), twf)), tiles_x);
  x1 = clamp_tile(__fadd_rn(floorf(__fdiv_rn(__fadd_rn(u, rx), twf)), 1.0f), tiles_x);
  y0 = clamp_tile(floorf(__fdiv_rn(__fsub_rn(v, ry), thf)), tiles_y);
  y1 = clamp_tile(__fadd_rn(floorf(__fdiv_rn(__fadd_rn(v, ry), thf)), 1.0f), tiles_y);
}

// packed rectangle: 4 x uint16 (x0, y0, x1, y1) in one uint2
__device__ __forceinline__ uint2 pack_rect(int x0, int y0, int x1, int y1) {
  return make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16),
                    (uint32_t)x1 | ((uint32_t)y1 << 16));
}
__device__ __forceinline__ void unpack_rect(uint2 r, int& x0, int& y0, int& x1,
                                            int& y1) {
  x0 = r.x & 0xFFFF;
  y0 = r.x >> 16;
  x1 = r.y & 0xFFFF;
  y1 = r.y >> 16;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace gftorf
