// render_pair.cu -- the line ratios (Algorithms 12-14) on the interleaved pair storage.
#include "render_impl.cuh"

namespace shw {

shw_status render_f32_pair(int mode, int interp, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                           cudaStream_t st)
{
    const float2 *p = static_cast<const float2 *>(v.data);
    const long long nvox = (long long)v.nx * v.ny * v.nz;
    if (nvox < (1LL << 31)) {
        SamplerF32Pair<int> s{p, v.nx, v.ny, v.nz, v.nx, v.nx * v.ny};
        return launch_render_modes<false>(mode, interp, s, s, cam, a, st);
    }
    SamplerF32Pair<long long> s{p, v.nx, v.ny, v.nz, (long long)v.nx, (long long)v.nx * v.ny};
    return launch_render_modes<false>(mode, interp, s, s, cam, a, st);
}

}  // namespace shw
