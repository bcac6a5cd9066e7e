// render_f16_big.cu -- marcher instances for f16 brick buffers of 2^31 elements or more
// (64-bit element offsets).
#include "render_impl.cuh"

namespace shw {

shw_status render_f16_big(int mode, int interp, const shw_volume &v, const shw_volume *v2,
                           const shw_camera &cam, const RenderArgs &a, cudaStream_t st)
{
    SamplerBrick<__half, long long> s{static_cast<const unsigned short *>(v.data), v.nx, v.ny, v.nz,
                                  ceil_div(v.nx, kBrick), ceil_div(v.ny, kBrick)};
    SamplerBrick<__half, long long> s2 = s;
    if (v2) s2.v = static_cast<const unsigned short *>(v2->data);
    return launch_render_modes<0>(mode, interp, s, s2, cam, a, st);
}

}  // namespace shw
