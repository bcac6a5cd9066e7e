// render_smooth_lat_b16.cu -- marcher instances for the in-ray box on the sample lattice (a
// step of 1/2 voxel, single-cube modes; Algorithm 8 as running sums), 16-bit bricks.
#include "render_impl.cuh"

namespace shw {

template <typename T>
static shw_status lat_bricks(int mode, int interp, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                             cudaStream_t st)
{
    SamplerBrick<T> s{static_cast<const unsigned short *>(v.data), v.nx, v.ny, v.nz, ceil_div(v.nx, kBrick),
                      ceil_div(v.ny, kBrick)};
    return launch_render_modes<2>(mode, interp, s, s, cam, a, st);
}

shw_status render_smooth_lat_b16(int mode, int interp, const shw_volume &v, const shw_camera &cam,
                                 const RenderArgs &a, cudaStream_t st)
{
    if (v.storage == SHW_BF16_BRICK) return lat_bricks<__nv_bfloat16>(mode, interp, v, cam, a, st);
    if (v.storage == SHW_F16_BRICK) return lat_bricks<__half>(mode, interp, v, cam, a, st);
    return SHW_EINVAL;
}

}  // namespace shw
