// render_f32.cu -- marcher instances for the linear float32 cube (< 2^31 voxels; larger
// cubes go to render_f32_big.cu's 64-bit-index instances).
#include "render_impl.cuh"

namespace shw {

shw_status render_f32(int mode, int interp, const shw_volume &v, const shw_volume *v2, const shw_camera &cam,
                      const RenderArgs &a, cudaStream_t st)
{
    const long long nvox = (long long)v.nx * v.ny * v.nz;
    if (nvox >= (1LL << 31)) return render_f32_big(mode, interp, v, v2, cam, a, st);
    SamplerF32<int> s{static_cast<const float *>(v.data), v.nx, v.ny, v.nz, v.nx, v.nx * v.ny};
    SamplerF32<int> s2 = s;
    if (v2) s2.v = static_cast<const float *>(v2->data);
    return launch_render_modes<0>(mode, interp, s, s2, cam, a, st);
}

}  // namespace shw
