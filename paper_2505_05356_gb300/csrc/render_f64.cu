// render_f64.cu -- double-precision instantiation of the compositing
// kernels (render_impl.cuh), used for gradient checks and tight parity.
#include "render_impl.cuh"

namespace gftorf {
template void launch_render_fwd<double>(const Layout&, const double*, double*,
                                        unsigned char*, cudaStream_t);
template void launch_render_bwd<double>(const Layout&, const double*,
                                        const double*, double*, unsigned char*,
                                        cudaStream_t);
}  // namespace gftorf
