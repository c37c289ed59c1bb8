// noalloc.cu -- gftorf_sort_footprints_noalloc: the binning of caller-given
// footprints with its scratch in a fixed device array instead of a
// caller-allocated workspace, for callers that cannot allocate device memory
// (see include/gftorf.h).
#include <mutex>

#include "gftorf_internal.cuh"

namespace gftorf {

bool binning_dims_ok(const gftorf_dims* d);
Layout binning_layout(const gftorf_dims* d);

namespace {

// Largest scratch this entry point can use; a device reserves it at the latest
// at the first call made there, and keeps it for the life of the process.
constexpr size_t kStaticScratchBytes = (size_t)32 << 20;  // 32 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once
// per device (host code may not use the symbol itself as a device pointer).
gftorf_status scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return GFTORF_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p)
      return GFTORF_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return GFTORF_OK;
}

}  // namespace
}  // namespace gftorf

using namespace gftorf;

extern "C" gftorf_status gftorf_sort_footprints_noalloc(
    const gftorf_dims* dims, const float* u, const float* v,
    const int32_t* radius, const float* z, uint64_t* keys, uint32_t* values,
    uint32_t* ranges, int64_t* count, void* stream) {
  if (!binning_dims_ok(dims)) return GFTORF_ERR_ARG;
  const Layout L = binning_layout(dims);
  if (L.N > 0 && (!u || !v || !radius || !z)) return GFTORF_ERR_ARG;
  if (!values || !ranges || !count) return GFTORF_ERR_ARG;
  if (L.total > kStaticScratchBytes) return GFTORF_ERR_WORKSPACE;
  unsigned char* ws = nullptr;
  gftorf_status s = scratch_for_current_device(&ws);
  if (s != GFTORF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: reset the status block
  cudaMemsetAsync(ws + L.off_header, 0, sizeof(Header), st);
  launch_footprints(L, u, v, radius, z, ws, st);
  launch_binning(L, ws, st);
  if (L.cap > 0)
    cudaMemcpyAsync(values, ws + L.off_values, (size_t)L.cap * 4, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(ranges, ws + L.off_ranges, (size_t)L.B * L.NT * sizeof(uint2),
                  cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(count, &at<Header>(ws, L.off_header)->count, sizeof(int64_t),
                  cudaMemcpyDeviceToDevice, st);
  if (keys) launch_export_keys(L, keys, ws, st);
  return cudaGetLastError() == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
}
