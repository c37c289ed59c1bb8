// render_f32.cu -- single-precision instantiation of the compositing
// kernels (render_impl.cuh).
#include "render_impl.cuh"

namespace gftorf {
template void launch_render_fwd<float>(const Layout&, const float*, float*,
                                       unsigned char*, cudaStream_t);
template void launch_render_bwd<float>(const Layout&, const float*, const float*,
                                       float*, unsigned char*, cudaStream_t);
}  // namespace gftorf
