// api.cu -- the C ABI of libgftorf: argument validation, workspace layout,
// and the launch sequence of each entry point (declared in include/gftorf.h).
#include <math.h>
#include <string.h>

#include <atomic>

#include "gftorf_internal.cuh"

namespace gftorf {

static std::atomic<int64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr double kLightSpeed = 299792458.0;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool tile_ok(int tw, int th) {
  return (tw == 8 && th == 8) || (tw == 16 && th == 16) || (tw == 16 && th == 32) ||
         (tw == 32 && th == 32) || (tw == 64 && th == 32) || (tw == 64 && th == 64);
}

bool dims_ok(const gftorf_dims* d) {
  if (!d) return false;
  // (depth-sort counts share a 32-bit status word with two flag bits)
  if (d->n_gaussians < 0 || d->n_gaussians >= (1 << 30)) return false;
  if (d->n_frames < 1 || d->n_frames > kMaxFrames) return false;
  if (d->width < 1 || d->height < 1 || d->width > 16384 || d->height > 16384) return false;
  if (!tile_ok(d->tile_w, d->tile_h)) return false;
  if (d->n_freq < 1 || d->n_freq > kMaxF || d->n_offsets < 1 || d->n_offsets > kMaxP)
    return false;
  if (d->dtype != GFTORF_F32 && d->dtype != GFTORF_F64) return false;
  if (d->render_mode != 0 && d->render_mode != 1) return false;
  const int ppt = d->pixels_per_thread;
  if (ppt != 0 && ppt != 1 && ppt != 2 && ppt != 4) return false;
  if (d->tile_w >= 32 && ppt != 0 && ppt != 4) return false;  // 32 wide or more: 4 per thread
  if (d->tile_w * d->tile_h / (ppt ? ppt : 2) < 32) return false;  // a full warp per tile
  if (d->flags & ~(GFTORF_FLAG_NO_TILE_CULL | GFTORF_FLAG_COUNT_PAIRS | GFTORF_FLAG_PHASOR |
                   GFTORF_FLAG_DEPTH))
    return false;
  if (d->n_sh != 0 && d->n_sh != 1 && d->n_sh != 4 && d->n_sh != 9 && d->n_sh != 16)
    return false;
  if (d->reserved != 0) return false;
  if (d->max_instances < 0 || d->max_instances > (int64_t)0xFFFFFFFFll) return false;
  // per-CTA tile counters ((tiles_x + 1) x (tiles_y + 1), 4 bytes each) live in
  // shared memory
  const int64_t corners = (int64_t)((d->width + d->tile_w - 1) / d->tile_w + 1) *
                          ((d->height + d->tile_h - 1) / d->tile_h + 1);
  if (corners > 50000) return false;
  return true;
}

// the parameter arrays the problem reads are present
bool params_ok(const Layout& L, const gftorf_gaussians* g) {
  if (L.N == 0) return true;
  if (!g->means || !g->scales || !g->quats || !g->opacity) return false;
  return L.nsh ? g->sh != nullptr : g->amplitude != nullptr;
}

Layout make_layout(const gftorf_dims* d) {
  Layout L;
  memset(&L, 0, sizeof(L));
  L.B = d->n_frames, L.N = d->n_gaussians, L.W = d->width, L.H = d->height;
  L.TW = d->tile_w, L.TH = d->tile_h, L.F = d->n_freq, L.P = d->n_offsets;
  L.C = L.F * L.P + 1, L.NF = 2 * L.F + 1, L.dtype = d->dtype;
  L.real_size = d->dtype == GFTORF_F64 ? 8 : 4;
  L.mode = d->render_mode;
  L.ppt = d->pixels_per_thread ? d->pixels_per_thread : (d->tile_w >= 32 ? 4 : 2);
  L.cull = (d->flags & GFTORF_FLAG_NO_TILE_CULL) ? 0 : 1;
  L.count_pairs = (d->flags & GFTORF_FLAG_COUNT_PAIRS) ? 1 : 0;
  L.phasor = (d->flags & GFTORF_FLAG_PHASOR) ? 1 : 0;
  L.depth = (d->flags & GFTORF_FLAG_DEPTH) ? 1 : 0;
  L.nsh = d->n_sh;
  L.C = L.F * L.P + 1 + (L.phasor ? 2 * L.F : 0) + (L.depth ? 1 : 0);
  L.tiles_x = (L.W + L.TW - 1) / L.TW;
  L.tiles_y = (L.H + L.TH - 1) / L.TH;
  L.NT = L.tiles_x * L.tiles_y;
  const int per16 = 16 / L.real_size;
  L.rec_stride = (8 + L.NF + per16 - 1) / per16 * per16;
  L.g2d_stride = 7 + L.NF;
  L.n_dblk = (L.N + kSortTile - 1) / kSortTile;
  L.n_chunk = (int)((d->max_instances + kChunk - 1) / kChunk) + L.B;
  L.n_scan = (int)(((size_t)L.B * L.N + kScanTile - 1) / kScanTile);
  int nw = 8;  // scatter warps: per-warp tile counters within 96 KB where possible
  while (nw > 1 && (size_t)nw * (L.tiles_x + 1) * (L.tiles_y + 1) * 4 > 96 * 1024) nw >>= 1;
  L.scatter_warps = nw;
  L.cap = d->max_instances;
  const size_t BN = (size_t)L.B * L.N, HW = (size_t)L.W * L.H;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at_ = o;
    o = align_up(o + bytes);
    return at_;
  };
  L.off_header = take(sizeof(Header));
  L.off_table = take(sizeof(Table) + sizeof(TableT<float>));
  L.off_rec = take(BN * L.rec_stride * L.real_size);
  L.off_rect = take(BN * sizeof(uint2));
  L.off_srect = take(BN * sizeof(uint2));
  L.off_zkey = take(BN * 4);
  L.off_zkey2 = take(2 * BN * 4);
  L.off_ids = take(BN * 4);
  L.off_ids2 = take(BN * 4);
  L.off_dhist = take(lb_bytes(L));
  L.off_dtot = take((size_t)L.B * 1024 * 4);
  L.off_ecnt = take((size_t)L.B * L.N * 4 + 4);
  L.off_bsum = take((size_t)(L.n_scan + 1) * 8);  // scan status words, 2 counters
  L.off_tcnt = take((size_t)L.n_chunk * L.NT * 4);
  L.off_toff = take((size_t)L.B * L.NT * 4);
  L.off_ranges = take((size_t)L.B * L.NT * sizeof(uint2));
  L.off_values = take((size_t)(L.cap > 0 ? L.cap : 1) * 4);
  L.off_tfinal = take((size_t)L.B * HW * L.real_size);
  L.off_nlast = take((size_t)L.B * HW * 4);
  L.off_g2d = take(BN * L.g2d_stride * L.real_size);
  L.total = o;
  return L;
}

gftorf_status check_ws(const Layout& L, void* ws, size_t bytes) {
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0 || bytes < L.total)
    return GFTORF_ERR_WORKSPACE;
  return GFTORF_OK;
}

gftorf_status launch_status() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
}

// Writes the batch table into the workspace from a kernel argument, so the
// upload is an ordinary kernel node inside a captured graph.
__global__ void store_table_kernel(Table t, Table* dst) {
  const int n = sizeof(Table) / sizeof(double);
  const double* s = reinterpret_cast<const double*>(&t);
  double* d = reinterpret_cast<double*>(dst);
  float* f = reinterpret_cast<float*>(dst + 1);  // TableT<float>: same fields
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    d[i] = s[i];
    f[i] = (float)s[i];
  }
}

bool finite(float x) { return isfinite(x) != 0; }

}  // namespace

// Workspace layout holding only the regions the binning stages touch (the
// projected records, per-pixel state and 2D-gradient regions are empty).
bool binning_dims_ok(const gftorf_dims* d) { return dims_ok(d); }

// Shape checks and channel layout for the optimisation-loop entry points.
bool train_dims_ok(const gftorf_dims* d) { return dims_ok(d); }
Layout train_layout(const gftorf_dims* d) { return make_layout(d); }

Layout binning_layout(const gftorf_dims* d) {
  Layout L = make_layout(d);
  const size_t BN = (size_t)L.B * L.N;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at_ = o;
    o = align_up(o + bytes);
    return at_;
  };
  L.off_header = take(sizeof(Header));
  L.off_table = take(0);
  L.off_rec = take(0);
  L.off_rect = take(BN * sizeof(uint2));
  L.off_srect = take(BN * sizeof(uint2));
  L.off_zkey = take(BN * 4);
  L.off_zkey2 = take(2 * BN * 4);
  L.off_ids = take(BN * 4);
  L.off_ids2 = take(BN * 4);
  L.off_dhist = take(lb_bytes(L));
  L.off_dtot = take((size_t)L.B * 1024 * 4);
  L.off_ecnt = take(BN * 4 + 4);
  L.off_bsum = take((size_t)(L.n_scan + 1) * 8);  // scan status words, 2 counters
  L.off_tcnt = take((size_t)L.n_chunk * L.NT * 4);
  L.off_toff = take((size_t)L.B * L.NT * 4);
  L.off_ranges = take((size_t)L.B * L.NT * sizeof(uint2));
  L.off_values = take((size_t)(L.cap > 0 ? L.cap : 1) * 4);
  L.off_tfinal = take(0);
  L.off_nlast = take(0);
  L.off_g2d = take(0);
  L.total = o;
  return L;
}

}  // namespace gftorf

using namespace gftorf;

extern "C" {

int32_t gftorf_version(void) { return 101; }

int64_t gftorf_kernel_launches(void) { return gftorf::launches_so_far(); }

gftorf_status gftorf_read_counters(const gftorf_dims* dims, void* workspace,
                                   size_t workspace_bytes, int64_t* counters,
                                   void* stream) {
  if (!dims_ok(dims) || !counters) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Header h;
  if (cudaMemcpyAsync(&h, static_cast<unsigned char*>(workspace) + L.off_header, sizeof(h),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GFTORF_ERR_CUDA;
  counters[0] = h.count;
  counters[1] = (int64_t)h.pairs;
  counters[2] = (int64_t)h.pairs_warp;
  return GFTORF_OK;
}

const char* gftorf_status_string(gftorf_status s) {
  switch (s) {
    case GFTORF_OK: return "ok";
    case GFTORF_ERR_ARG: return "invalid argument";
    case GFTORF_ERR_CAPACITY: return "tile-instance capacity exceeded";
    case GFTORF_ERR_TIMEOUT: return "bounded device wait timed out";
    case GFTORF_ERR_CUDA: return "CUDA error";
    case GFTORF_ERR_UNSUPPORTED: return "unsupported configuration";
    case GFTORF_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
  }
  return "unknown status";
}

size_t gftorf_workspace_size(const gftorf_dims* dims) {
  if (!dims_ok(dims)) return 0;
  return make_layout(dims).total;
}

gftorf_status gftorf_preprocess(const gftorf_dims* dims,
                                const gftorf_gaussians* g,
                                const gftorf_frame* frames,
                                const gftorf_sensor* sensor,
                                const gftorf_consts* consts, void* workspace,
                                size_t workspace_bytes, void* stream) {
  gftorf::TraceRange trace_("gftorf_preprocess");
  if (!dims_ok(dims) || !g || !frames || !sensor || !consts) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  if (!params_ok(L, g)) return GFTORF_ERR_ARG;
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  Table t;
  memset(&t, 0, sizeof(t));
  for (int b = 0; b < L.B; ++b) {
    const gftorf_frame& f = frames[b];
    if (!(f.fx > 0) || !(f.fy > 0) || !finite(f.cx) || !finite(f.cy) ||
        !(f.near_plane > 0) || !finite(f.near_plane) || !finite(f.time) ||
        !finite(f.phase_offset_rad) || !finite(f.interp_t0) || !finite(f.interp_t1) ||
        f.interp_t0 > f.interp_t1)
      return GFTORF_ERR_ARG;
    for (int k = 0; k < 12; ++k)
      if (!finite(f.world_to_cam[k])) return GFTORF_ERR_ARG;
    FrameT<double>& d = t.fr[b];
    d.fx = f.fx, d.fy = f.fy, d.cx = f.cx, d.cy = f.cy;
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) d.R[3 * r + c] = f.world_to_cam[4 * r + c];
      d.t[r] = f.world_to_cam[4 * r + 3];
    }
    for (int c = 0; c < 3; ++c)
      d.o[c] = -(d.R[c] * d.t[0] + d.R[3 + c] * d.t[1] + d.R[6 + c] * d.t[2]);
    d.near_plane = f.near_plane, d.time = f.time;
    // c_k multiplies t^k, or under Eq. 7 the interpolation of t0^k and t1^k
    const double tt = f.time, t0 = f.interp_t0, t1 = f.interp_t1;
    double p0 = 1, p1 = 1, pt = 1;
    for (int k = 0; k < 3; ++k) {
      p0 *= t0, p1 *= t1, pt *= tt;
      d.tp[k] = t1 > t0 ? ((t1 - tt) * p0 + (tt - t0) * p1) / (t1 - t0) : pt;
    }
    for (int j = 0; j < L.P; ++j) {
      const double phi = (double)sensor->offset_rad[j] + (double)f.phase_offset_rad;
      d.cos_off[j] = cos(phi);
      d.sin_off[j] = sin(phi);
    }
    d.limx = (double)consts->guard * 0.5 * L.W / f.fx;
    d.limy = (double)consts->guard * 0.5 * L.H / f.fy;
  }
  for (int k = 0; k < L.F; ++k) {
    if (!finite(sensor->freq_hz[k]) || sensor->freq_hz[k] < 0) return GFTORF_ERR_ARG;
    t.kf[k] = 4.0 * (double)sensor->freq_hz[k] / kLightSpeed;
  }
  for (int j = 0; j < L.P; ++j)
    if (!finite(sensor->offset_rad[j])) return GFTORF_ERR_ARG;
  if (!finite(sensor->source_intensity)) return GFTORF_ERR_ARG;
  t.source = sensor->source_intensity;
  if (!(consts->dilation >= 0) || !(consts->alpha_max > 0) || !(consts->alpha_max <= 1) ||
      !(consts->alpha_min >= 0) || !(consts->t_min >= 0) || !(consts->guard > 0) ||
      !(consts->sigma_cut > 0))
    return GFTORF_ERR_ARG;
  t.dilation = consts->dilation, t.alpha_max = consts->alpha_max;
  t.alpha_min = consts->alpha_min, t.t_min = consts->t_min;
  t.sigma_cut = consts->sigma_cut;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  cudaMemsetAsync(ws + L.off_header, 0, sizeof(Header), st);
  store_table_kernel<<<1, 256, 0, st>>>(t, at<Table>(ws, L.off_table));
  count_launches(1);
  if (L.dtype == GFTORF_F32)
    launch_preprocess<float>(L, *g, ws, st);
  else
    launch_preprocess<double>(L, *g, ws, st);
  return launch_status();
}

gftorf_status gftorf_bin(const gftorf_dims* dims, void* workspace,
                         size_t workspace_bytes, void* stream) {
  gftorf::TraceRange trace_("gftorf_bin");
  if (!dims_ok(dims)) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  launch_binning(L, static_cast<unsigned char*>(workspace), static_cast<cudaStream_t>(stream));
  return launch_status();
}

gftorf_status gftorf_composite_fwd(const gftorf_dims* dims, const void* bg,
                                   void* out, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  gftorf::TraceRange trace_("gftorf_composite_fwd");
  if (!dims_ok(dims) || !bg || !out) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  if (L.dtype == GFTORF_F32)
    launch_render_fwd<float>(L, static_cast<const float*>(bg), static_cast<float*>(out), ws, st);
  else
    launch_render_fwd<double>(L, static_cast<const double*>(bg), static_cast<double*>(out), ws,
                              st);
  return launch_status();
}

gftorf_status gftorf_render_fwd(const gftorf_dims* dims, const void* bg,
                                void* out, void* workspace,
                                size_t workspace_bytes, void* stream) {
  gftorf::TraceRange trace_("gftorf_render_fwd");
  if (!dims_ok(dims) || !bg || !out) return GFTORF_ERR_ARG;
  gftorf_status s = gftorf_bin(dims, workspace, workspace_bytes, stream);
  if (s != GFTORF_OK) return s;
  return gftorf_composite_fwd(dims, bg, out, workspace, workspace_bytes, stream);
}

gftorf_status gftorf_zero_grad_buffers(const gftorf_dims* dims,
                                       const gftorf_gradients* grads,
                                       void* workspace, size_t workspace_bytes,
                                       void* stream) {
  gftorf::TraceRange trace_("gftorf_zero_grad_buffers");
  if (!dims_ok(dims) || !grads) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  cudaMemsetAsync(ws + L.off_g2d, 0, (size_t)L.B * L.N * L.g2d_stride * L.real_size, st);
  if (grads->bg) cudaMemsetAsync(grads->bg, 0, (size_t)L.B * L.C * L.real_size, st);
  return launch_status();
}

gftorf_status gftorf_composite_bwd(const gftorf_dims* dims, const void* bg,
                                   const void* dL_dout,
                                   const gftorf_gradients* grads,
                                   void* workspace, size_t workspace_bytes,
                                   void* stream) {
  gftorf::TraceRange trace_("gftorf_composite_bwd");
  if (!dims_ok(dims) || !bg || !dL_dout || !grads) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  if (L.dtype == GFTORF_F32)
    launch_render_bwd<float>(L, static_cast<const float*>(bg),
                             static_cast<const float*>(dL_dout),
                             static_cast<float*>(grads->bg), ws, st);
  else
    launch_render_bwd<double>(L, static_cast<const double*>(bg),
                              static_cast<const double*>(dL_dout),
                              static_cast<double*>(grads->bg), ws, st);
  return launch_status();
}

gftorf_status gftorf_preprocess_bwd(const gftorf_dims* dims,
                                    const gftorf_gaussians* g,
                                    const gftorf_gradients* grads,
                                    void* workspace, size_t workspace_bytes,
                                    void* stream) {
  gftorf::TraceRange trace_("gftorf_preprocess_bwd");
  if (!dims_ok(dims) || !g || !grads) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  if (!params_ok(L, g)) return GFTORF_ERR_ARG;
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  if (L.dtype == GFTORF_F32)
    launch_preprocess_bwd<float>(L, *g, *grads, ws, st);
  else
    launch_preprocess_bwd<double>(L, *g, *grads, ws, st);
  return launch_status();
}

gftorf_status gftorf_render_bwd(const gftorf_dims* dims,
                                const gftorf_gaussians* g, const void* bg,
                                const void* dL_dout,
                                const gftorf_gradients* grads, void* workspace,
                                size_t workspace_bytes, void* stream) {
  gftorf::TraceRange trace_("gftorf_render_bwd");
  if (!dims_ok(dims) || !g || !bg || !dL_dout || !grads) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  if (!params_ok(L, g)) return GFTORF_ERR_ARG;
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  s = gftorf_zero_grad_buffers(dims, grads, workspace, workspace_bytes, stream);
  if (s != GFTORF_OK) return s;
  s = gftorf_composite_bwd(dims, bg, dL_dout, grads, workspace, workspace_bytes, stream);
  if (s != GFTORF_OK) return s;
  return gftorf_preprocess_bwd(dims, g, grads, workspace, workspace_bytes, stream);
}

gftorf_status gftorf_sort_footprints(const gftorf_dims* dims, const float* u,
                                     const float* v, const int32_t* radius,
                                     const float* z, uint64_t* keys,
                                     uint32_t* values, uint32_t* ranges,
                                     int64_t* count, void* workspace,
                                     size_t workspace_bytes, void* stream) {
  gftorf::TraceRange trace_("gftorf_sort_footprints");
  if (!dims_ok(dims)) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  if (L.N > 0 && (!u || !v || !radius || !z)) return GFTORF_ERR_ARG;
  if (!values || !ranges || !count) return GFTORF_ERR_ARG;
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  cudaMemsetAsync(ws + L.off_header, 0, sizeof(Header), st);
  launch_footprints(L, u, v, radius, z, ws, st);
  launch_binning(L, ws, st);
  return gftorf_export_tile_lists(dims, keys, values, ranges, count, workspace,
                                  workspace_bytes, stream);
}

gftorf_status gftorf_export_tile_lists(const gftorf_dims* dims, uint64_t* keys,
                                       uint32_t* values, uint32_t* ranges,
                                       int64_t* count, void* workspace,
                                       size_t workspace_bytes, void* stream) {
  if (!dims_ok(dims) || !values || !ranges || !count) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  if (L.cap > 0)
    cudaMemcpyAsync(values, ws + L.off_values, (size_t)L.cap * 4, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(ranges, ws + L.off_ranges, (size_t)L.B * L.NT * sizeof(uint2),
                  cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(count, &at<Header>(ws, L.off_header)->count, sizeof(int64_t),
                  cudaMemcpyDeviceToDevice, st);
  if (keys) launch_export_keys(L, keys, ws, st);
  return launch_status();
}

gftorf_status gftorf_export_pixel_state(const gftorf_dims* dims, void* t_final,
                                        uint32_t* n_last, void* workspace,
                                        size_t workspace_bytes, void* stream) {
  if (!dims_ok(dims)) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  const size_t px = (size_t)L.B * L.W * L.H;
  if (t_final)
    cudaMemcpyAsync(t_final, ws + L.off_tfinal, px * L.real_size, cudaMemcpyDeviceToDevice, st);
  if (n_last)
    cudaMemcpyAsync(n_last, ws + L.off_nlast, px * 4, cudaMemcpyDeviceToDevice, st);
  return launch_status();
}

gftorf_status gftorf_read_device_status(const gftorf_dims* dims, void* workspace,
                                        size_t workspace_bytes, int64_t* count,
                                        void* stream) {
  if (!dims_ok(dims)) return GFTORF_ERR_ARG;
  const Layout L = make_layout(dims);
  gftorf_status s = check_ws(L, workspace, workspace_bytes);
  if (s != GFTORF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Header h;
  if (cudaMemcpyAsync(&h, static_cast<unsigned char*>(workspace) + L.off_header, sizeof(h),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GFTORF_ERR_CUDA;
  if (count) *count = h.count;
  return (gftorf_status)h.status;
}

}  // extern "C"
