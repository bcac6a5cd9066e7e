// render_axis_fix.cu -- the plane-sweep kernels with the fixed 72 x 21 staged box (a separate translation
// unit so that the two families compile in parallel).
#include "render_axis.cuh"

namespace shw {

template shw_status launch_axis<true>(int, int, bool, const CUtensorMap &, const float *, const shw_camera &,
                                    const RenderArgs &, const AxisArgs &, unsigned, size_t, cudaStream_t);

}  // namespace shw
