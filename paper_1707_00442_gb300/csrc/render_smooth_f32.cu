// render_smooth_f32.cu -- marcher instances with in-ray smoothing (Algorithms 8-9) for
// the linear float32 cube.
#include "render_impl.cuh"

namespace shw {

shw_status render_smooth_f32(int mode, int interp, const shw_volume &v, const shw_volume *v2,
                             const shw_camera &cam, const RenderArgs &a, cudaStream_t st)
{
    const long long nvox = (long long)v.nx * v.ny * v.nz;
    if (nvox < (1LL << 31)) {
        SamplerF32<int> s{static_cast<const float *>(v.data), v.nx, v.ny, v.nz, v.nx, v.nx * v.ny};
        SamplerF32<int> s2 = s;
        if (v2) s2.v = static_cast<const float *>(v2->data);
        return launch_render_modes<1>(mode, interp, s, s2, cam, a, st);
    }
    SamplerF32<long long> s{static_cast<const float *>(v.data), v.nx, v.ny, v.nz, (long long)v.nx,
                            (long long)v.nx * v.ny};
    SamplerF32<long long> s2 = s;
    if (v2) s2.v = static_cast<const float *>(v2->data);
    return launch_render_modes<1>(mode, interp, s, s2, cam, a, st);
}

}  // namespace shw
