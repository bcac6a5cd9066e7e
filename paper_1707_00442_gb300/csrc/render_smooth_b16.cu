// render_smooth_b16.cu -- marcher instances with in-ray smoothing (Algorithms 8-9) for the
// bf16 and fp16 brick storages.
#include "render_impl.cuh"

namespace shw {

template <typename T>
static shw_status smooth_bricks(int mode, int interp, const shw_volume &v, const shw_volume *v2,
                                const shw_camera &cam, const RenderArgs &a, cudaStream_t st)
{
    SamplerBrick<T> s{static_cast<const unsigned short *>(v.data), v.nx, v.ny, v.nz, ceil_div(v.nx, kBrick),
                      ceil_div(v.ny, kBrick)};
    SamplerBrick<T> s2 = s;
    if (v2) s2.v = static_cast<const unsigned short *>(v2->data);
    return launch_render_modes<1>(mode, interp, s, s2, cam, a, st);
}

shw_status render_smooth_b16(int mode, int interp, const shw_volume &v, const shw_volume *v2,
                             const shw_camera &cam, const RenderArgs &a, cudaStream_t st)
{
    if (v.storage == SHW_BF16_BRICK) return smooth_bricks<__nv_bfloat16>(mode, interp, v, v2, cam, a, st);
    if (v.storage == SHW_F16_BRICK) return smooth_bricks<__half>(mode, interp, v, v2, cam, a, st);
    return SHW_EINVAL;
}

}  // namespace shw
