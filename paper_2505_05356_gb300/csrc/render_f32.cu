// render_f32.cu -- instantiation of the compositing kernels (render_impl.cuh)
// for float.
#include "render_impl.cuh"

namespace gftorf {
template void launch_render_fwd_t<float, false>(const Layout&, const float*, float*, unsigned char*,
                                         cudaStream_t);
template void launch_render_bwd_t<float, false>(const Layout&, const float*, const float*, float*,
                                         unsigned char*, cudaStream_t);
}  // namespace gftorf
