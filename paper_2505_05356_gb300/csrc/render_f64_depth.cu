// render_f64_depth.cu -- instantiation of the compositing kernels (render_impl.cuh)
// for double with the Eq. 5 mean-depth channel.
#include "render_impl.cuh"

namespace gftorf {
template void launch_render_fwd_t<double, true>(const Layout&, const double*, double*, unsigned char*,
                                         cudaStream_t);
template void launch_render_bwd_t<double, true>(const Layout&, const double*, const double*, double*,
                                         unsigned char*, cudaStream_t);
}  // namespace gftorf
