// render_slab_h16.cu -- the staged marcher's instances for the linear 16-bit storages
// (bfloat16 and binary16 cubes, and the line ratios' 16-bit pairs); FP32 interpolation
// and accumulation, as for every storage.
#include "render_slab.cuh"

namespace shw {

shw_status render_slab_h16(int mode, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                           cudaStream_t st)
{
    const int sy = v.nx, sz = v.nx * v.ny;
    switch (v.storage) {
    case SHW_BF16: {
        const SamplerLin16<__nv_bfloat16> s{static_cast<const unsigned short *>(v.data), v.nx, v.ny, v.nz, sy, sz};
        return slab_launch<ElemH<__nv_bfloat16>>(mode, s, v.data, cam, a, st);
    }
    case SHW_F16: {
        const SamplerLin16<__half> s{static_cast<const unsigned short *>(v.data), v.nx, v.ny, v.nz, sy, sz};
        return slab_launch<ElemH<__half>>(mode, s, v.data, cam, a, st);
    }
    case SHW_BF16_PAIR: {
        const SamplerLin16Pair<__nv_bfloat16> s{static_cast<const unsigned *>(v.data), v.nx, v.ny, v.nz, sy, sz};
        return slab_launch<ElemHPair<__nv_bfloat16>>(mode, s, v.data, cam, a, st);
    }
    case SHW_F16_PAIR: {
        const SamplerLin16Pair<__half> s{static_cast<const unsigned *>(v.data), v.nx, v.ny, v.nz, sy, sz};
        return slab_launch<ElemHPair<__half>>(mode, s, v.data, cam, a, st);
    }
    default: return SHW_EUNSUPPORTED;
    }
}

}  // namespace shw
