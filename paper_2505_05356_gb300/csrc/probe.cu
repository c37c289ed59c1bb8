// probe.cu -- throughput probes of the two pipes that bound the compositing
// kernels (each evaluated (pixel, Gaussian) pair of Eq. 4 / Eq. S3 is a short
// chain of FP32 multiply-adds around one base-2 exponential): a loop of
// independent FP32 fused multiply-adds, and a loop of independent
// ex2.approx.ftz.f32 evaluations on the multi-function unit.  The measured
// rates are the denominators of those kernels' rooflines.
#include "gftorf_internal.cuh"

namespace gftorf {
namespace {

constexpr int kChains = 8;          // independent dependency chains per thread
constexpr int kProbeThreads = 256;  // 8 CTAs of 256 threads fill an SM (64 warps)
constexpr int kUnroll = 16;

// x <- x a + b on kChains chains; a, b are kernel arguments, so nothing folds
__global__ void __launch_bounds__(kProbeThreads) ffma_probe_kernel(float* sink, int iters,
                                                                   float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k);
  for (int i = 0; i < iters; i += kUnroll) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = __fmaf_rn(x[k], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0f) sink[0] = s;  // keeps the loop live; never true for a, b > 0
}

// x <- 2^(-x): bounded chains (they settle near 0.64) of dependent ex2 calls
__global__ void __launch_bounds__(kProbeThreads) ex2_probe_kernel(float* sink, int iters) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 0.01f * (float)(threadIdx.x + k);
  for (int i = 0; i < iters; i += kUnroll) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = ex2_approx(-x[k]);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0f) sink[0] = s;  // never true: 2^-x > 0
}

}  // namespace
}  // namespace gftorf

using namespace gftorf;

extern "C" gftorf_status gftorf_probe_throughput(int32_t kind, int32_t iters, float* sink,
                                                 int64_t* lane_ops, void* stream) {
  if ((kind != GFTORF_PROBE_FFMA && kind != GFTORF_PROBE_EX2) || iters < kUnroll ||
      iters % kUnroll != 0 || !sink || !lane_ops)
    return GFTORF_ERR_ARG;
  const int blocks = sm_count() * 8;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (kind == GFTORF_PROBE_FFMA)
    ffma_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(sink, iters, 0.999f, 1e-3f);
  else
    ex2_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(sink, iters);
  count_launches(1);
  *lane_ops = (int64_t)blocks * kProbeThreads * kChains * (int64_t)iters;
  return cudaGetLastError() == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
}
