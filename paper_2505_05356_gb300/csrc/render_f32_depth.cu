// render_f32_depth.cu -- instantiation of the compositing kernels (render_impl.cuh)
// for float with the Eq. 5 mean-depth channel.
#include "render_impl.cuh"

namespace gftorf {
template void launch_render_fwd_t<float, true>(const Layout&, const float*, float*, unsigned char*,
                                         cudaStream_t);
template void launch_render_bwd_t<float, true>(const Layout&, const float*, const float*, float*,
                                         unsigned char*, cudaStream_t);
}  // namespace gftorf
