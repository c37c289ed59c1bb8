// train.cu -- the optimisation-loop steps around the renderer: the random
// background drawn per iteration, the raw-sample L2 loss with its gradient,
// and a multi-group projected Adam update (Sec. 4: raw-quad loss, Adam with
// betas (0.9, 0.999) and epsilon 1e-15, a fresh background U(-1, 1) every
// iteration).  Every kernel reads its iteration number from the device-side
// state, so a whole iteration can be captured once and replayed.
#include <cmath>
#include <cstring>

#include "gftorf_internal.cuh"

namespace gftorf {

bool train_dims_ok(const gftorf_dims* d);
Layout train_layout(const gftorf_dims* d);

namespace {

constexpr int kBgMax = 65536;

// SplitMix64 (Steele, Lea, Flood 2014): the k-th output of the generator
// seeded with s is mix(s + k * 0x9E3779B97F4A7C15).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// values [offset, offset + n_bg) of the iteration's `stride` background
// values (a shard of frames draws its own slice of the whole batch's)
__global__ void __launch_bounds__(256)
    train_begin_kernel(gftorf_train_state* st, float* bg, int n_bg, uint64_t seed,
                       uint64_t offset, uint64_t stride) {
  __shared__ int64_t s_step;
  if (threadIdx.x == 0) {
    s_step = st->step + 1;
    st->step = s_step;
    st->loss = 0.0;
  }
  __syncthreads();
  if (!bg) return;
  const uint64_t base = (uint64_t)(s_step - 1) * stride + offset + 1;
  for (int i = threadIdx.x; i < n_bg; i += blockDim.x) {
    const uint32_t top = (uint32_t)(splitmix64_at(seed, base + i) >> 40);  // 24 bits
    // 2 u - 1 with u = top 2^-24: exact in single precision
    bg[i] = (float)top * 0x1.0p-23f - 1.0f;
  }
}

// out/target/grad are [B][C][HW]; raw channels are c < FP.  With vec (HW a
// multiple of 4, 16-byte aligned arrays) each thread takes float4 groups of
// pixels, else single values.
__global__ void __launch_bounds__(256)
    l2_loss_kernel(const float* __restrict__ out, const float* __restrict__ target,
                   float* __restrict__ grad, gftorf_train_state* st, int64_t n_rows,
                   int C, int FP, int64_t HW, float scale, double inv_m, int vec) {
  float part = 0.f;
  if (vec) {
    const int64_t HW4 = HW >> 2;
    const int64_t total = n_rows * HW4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t row = e / HW4;
      const int c = (int)(row % C);
      float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c < FP) {
        const float4 o = reinterpret_cast<const float4*>(out)[e];
        const float4 t = __ldcs(reinterpret_cast<const float4*>(target) + e);
        const float rx = o.x - t.x, ry = o.y - t.y, rz = o.z - t.z, rw = o.w - t.w;
        part += rx * rx + ry * ry + rz * rz + rw * rw;
        g = make_float4(scale * rx, scale * ry, scale * rz, scale * rw);
      }
      reinterpret_cast<float4*>(grad)[e] = g;
    }
  } else {
    const int64_t total = n_rows * HW;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int c = (int)((e / HW) % C);
      float g = 0.f;
      if (c < FP) {
        const float r = out[e] - target[e];
        part += r * r;
        g = scale * r;
      }
      grad[e] = g;
    }
  }
  // block sum in double, one atomic per CTA
  double d = part;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  __shared__ double s_part[8];
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_part[w];
    if (sum != 0.0) atomicAdd(&st->loss, sum * inv_m);
  }
}

struct AdamArgs {
  gftorf_adam_group g[GFTORF_MAX_ADAM_GROUPS];
  int n;
  float b1, b2, eps;
};

__global__ void __launch_bounds__(256)
    adam_kernel(AdamArgs a, const gftorf_train_state* __restrict__ st) {
  const int64_t t = st->step > 0 ? st->step : 1;
  const float bc1 = 1.f - powf(a.b1, (float)t);
  const float bc2 = 1.f - powf(a.b2, (float)t);
  const float ib1 = 1.f / bc1, ib2 = 1.f / bc2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int k = 0; k < a.n; ++k) {
    const gftorf_adam_group G = a.g[k];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < G.n; i += stride) {
      const float g = G.grad[i];
      const float m = a.b1 * G.m[i] + (1.f - a.b1) * g;
      const float v = a.b2 * G.v[i] + (1.f - a.b2) * g * g;
      G.m[i] = m;
      G.v[i] = v;
      const float step = G.lr * (m * ib1) / (sqrtf(v * ib2) + a.eps);
      G.param[i] = fminf(G.hi, fmaxf(G.lo, G.param[i] - step));
    }
  }
}

gftorf_status last_status() {
  return cudaGetLastError() == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
}

}  // namespace
}  // namespace gftorf

using namespace gftorf;

extern "C" gftorf_status gftorf_train_begin_shard(gftorf_train_state* state, float* bg,
                                                  int64_t n_bg, uint64_t seed,
                                                  int64_t bg_offset, int64_t bg_stride,
                                                  void* stream) {
  gftorf::TraceRange trace_("gftorf_train_begin");
  if (!state || n_bg < 0 || n_bg > kBgMax || bg_offset < 0 || bg_offset + n_bg > bg_stride ||
      bg_stride > ((int64_t)1 << 40))
    return GFTORF_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(state) & 7) != 0) return GFTORF_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  train_begin_kernel<<<1, 256, 0, st>>>(state, n_bg ? bg : nullptr, (int)n_bg, seed,
                                        (uint64_t)bg_offset, (uint64_t)bg_stride);
  count_launches(1);
  return last_status();
}

extern "C" gftorf_status gftorf_train_begin(gftorf_train_state* state, float* bg, int64_t n_bg,
                                            uint64_t seed, void* stream) {
  return gftorf_train_begin_shard(state, bg, n_bg, seed, 0, n_bg > 0 ? n_bg : 0, stream);
}

extern "C" gftorf_status gftorf_l2_loss_scaled(const gftorf_dims* dims, const float* out,
                                               const float* target, float* dL_dout,
                                               gftorf_train_state* state, double count,
                                               void* stream) {
  gftorf::TraceRange trace_("gftorf_l2_loss");
  if (!train_dims_ok(dims) || dims->dtype != GFTORF_F32 || !out || !target || !dL_dout ||
      !state || !(count >= 1.0) || !std::isfinite(count))
    return GFTORF_ERR_ARG;
  const Layout L = train_layout(dims);
  const int64_t HW = (int64_t)L.W * L.H;
  const int64_t n_rows = (int64_t)L.B * L.C;
  const int FP = L.F * L.P;
  const double M = count;
  const bool vec = (HW & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(target) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(dL_dout) & 15) == 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  l2_loss_kernel<<<sm_count() * 8, 256, 0, st>>>(out, target, dL_dout, state, n_rows, L.C, FP,
                                                 HW, (float)(2.0 / M), 1.0 / M, vec ? 1 : 0);
  count_launches(1);
  return last_status();
}

extern "C" gftorf_status gftorf_l2_loss(const gftorf_dims* dims, const float* out,
                                        const float* target, float* dL_dout,
                                        gftorf_train_state* state, void* stream) {
  if (!train_dims_ok(dims)) return GFTORF_ERR_ARG;
  const Layout L = train_layout(dims);
  const double M = (double)L.B * (L.F * L.P) * ((double)L.W * L.H);
  return gftorf_l2_loss_scaled(dims, out, target, dL_dout, state, M, stream);
}

extern "C" gftorf_status gftorf_adam_step(const gftorf_adam_group* groups, int n_groups,
                                          float beta1, float beta2, float eps,
                                          const gftorf_train_state* state, void* stream) {
  gftorf::TraceRange trace_("gftorf_adam_step");
  if (!groups || n_groups < 0 || n_groups > GFTORF_MAX_ADAM_GROUPS || !state)
    return GFTORF_ERR_ARG;
  if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
    return GFTORF_ERR_ARG;
  AdamArgs a;
  memset(&a, 0, sizeof(a));
  int64_t most = 0;
  for (int k = 0; k < n_groups; ++k) {
    const gftorf_adam_group& G = groups[k];
    if (G.n < 0 || (G.n > 0 && (!G.param || !G.grad || !G.m || !G.v))) return GFTORF_ERR_ARG;
    if (!(G.lo <= G.hi) || !std::isfinite(G.lr)) return GFTORF_ERR_ARG;
    a.g[k] = G;
    most = G.n > most ? G.n : most;
  }
  a.n = n_groups, a.b1 = beta1, a.b2 = beta2, a.eps = eps;
  if (most == 0) return GFTORF_OK;
  const int64_t want = (most + 255) / 256;
  const int blocks = (int)(want < (int64_t)sm_count() * 8 ? want : (int64_t)sm_count() * 8);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  adam_kernel<<<blocks, 256, 0, st>>>(a, state);
  count_launches(1);
  return last_status();
}
