// render_pair.cu -- the line ratios (Algorithms 12-14) on the interleaved pair storages
// (float32 pairs and 16-bit pair bricks).
#include "render_impl.cuh"

namespace shw {

shw_status render_f32_pair(int mode, int interp, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                           cudaStream_t st)
{
    const float2 *p = static_cast<const float2 *>(v.data);
    const long long nvox = (long long)v.nx * v.ny * v.nz;
    if (nvox < (1LL << 31)) {
        SamplerF32Pair<int> s{p, v.nx, v.ny, v.nz, v.nx, v.nx * v.ny};
        return launch_render_modes<0>(mode, interp, s, s, cam, a, st);
    }
    SamplerF32Pair<long long> s{p, v.nx, v.ny, v.nz, (long long)v.nx, (long long)v.nx * v.ny};
    return launch_render_modes<0>(mode, interp, s, s, cam, a, st);
}

template <typename T>
static shw_status render_bricks_pair(int mode, int interp, const shw_volume &v, const shw_camera &cam,
                                     const RenderArgs &a, cudaStream_t st)
{
    const unsigned *p = static_cast<const unsigned *>(v.data);
    const int nbx = ceil_div(v.nx, kBrick), nby = ceil_div(v.ny, kBrick);
    const long long elems = (long long)nbx * nby * ceil_div(v.nz, kBrick) * kBrickElems;
    if (elems < (1LL << 31)) {  // 32-bit element offsets
        SamplerBrickPair<T, int> s{p, v.nx, v.ny, v.nz, nbx, nby};
        return launch_render_modes<0>(mode, interp, s, s, cam, a, st);
    }
    SamplerBrickPair<T, long long> s{p, v.nx, v.ny, v.nz, nbx, nby};
    return launch_render_modes<0>(mode, interp, s, s, cam, a, st);
}

shw_status render_pair(int mode, int interp, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                       cudaStream_t st)
{
    switch (v.storage) {
    case SHW_F32_PAIR: return render_f32_pair(mode, interp, v, cam, a, st);
    case SHW_BF16_PAIR_BRICK: return render_bricks_pair<__nv_bfloat16>(mode, interp, v, cam, a, st);
    case SHW_F16_PAIR_BRICK: return render_bricks_pair<__half>(mode, interp, v, cam, a, st);
    default: return SHW_EINVAL;
    }
}

}  // namespace shw
