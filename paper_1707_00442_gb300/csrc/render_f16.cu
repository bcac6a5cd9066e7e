// render_f16.cu -- marcher instances for the f16 brick storage (32^3 bricks + apron),
// 32-bit element offsets; buffers of 2^31 elements or more go to render_f16_big.cu.
#include "render_impl.cuh"

namespace shw {

shw_status render_f16(int mode, int interp, const shw_volume &v, const shw_volume *v2, const shw_camera &cam,
                      const RenderArgs &a, cudaStream_t st)
{
    const long long elems = (long long)ceil_div(v.nx, kBrick) * ceil_div(v.ny, kBrick) * ceil_div(v.nz, kBrick) *
                            kBrickElems;
    if (elems >= (1LL << 31)) return render_f16_big(mode, interp, v, v2, cam, a, st);
    SamplerBrick<__half, int> s{static_cast<const unsigned short *>(v.data), v.nx, v.ny, v.nz, ceil_div(v.nx, kBrick),
                            ceil_div(v.ny, kBrick)};
    SamplerBrick<__half, int> s2 = s;
    if (v2) s2.v = static_cast<const unsigned short *>(v2->data);
    return launch_render_modes<0>(mode, interp, s, s2, cam, a, st);
}

}  // namespace shw
