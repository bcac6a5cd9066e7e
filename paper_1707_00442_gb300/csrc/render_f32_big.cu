// render_f32_big.cu -- marcher instances for linear float32 cubes of 2^31 voxels or more
// (64-bit element offsets).
#include "render_impl.cuh"

namespace shw {

shw_status render_f32_big(int mode, int interp, const shw_volume &v, const shw_volume *v2, const shw_camera &cam,
                          const RenderArgs &a, cudaStream_t st)
{
    SamplerF32<long long> s{static_cast<const float *>(v.data), v.nx, v.ny, v.nz, (long long)v.nx,
                            (long long)v.nx * v.ny};
    SamplerF32<long long> s2 = s;
    if (v2) s2.v = static_cast<const float *>(v2->data);
    return launch_render_modes<0>(mode, interp, s, s2, cam, a, st);
}

}  // namespace shw
