// render_axis_var.cu -- the plane-sweep kernels with a staged box sized per launch (a separate translation
// unit so that the two families compile in parallel).
#include "render_axis.cuh"

namespace shw {

template shw_status launch_axis<false>(int, int, bool, const CUtensorMap &, const float *, const shw_camera &,
                                    const RenderArgs &, const AxisArgs &, unsigned, size_t, cudaStream_t);

}  // namespace shw
