// render_slab.cu -- the staged marcher's dispatch and its float32 instances (the cube, and
// the line ratios' interleaved pair storage); the linear 16-bit storages are instanced in
// render_slab_h16.cu.
#include "render_slab.cuh"

namespace shw {

shw_status render_slab(int mode, int interp, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                       cudaStream_t st)
{
    if (interp != SHW_TRILINEAR || a.smooth != SHW_SMOOTH_NONE || debug(SHW_DEBUG_NO_STAGING))
        return SHW_EUNSUPPORTED;
    if ((long long)v.nx * v.ny * v.nz >= (1LL << 31) || v.nx < 2 || v.ny < 2 || v.nz < 2 || !aligned(v.data, 16))
        return SHW_EUNSUPPORTED;
    const bool ratio = mode == SHW_RATIO || mode == SHW_RATIO_MIP;
    switch (v.storage) {
    case SHW_F32: {
        if (ratio || v.nx % 4 != 0) return SHW_EUNSUPPORTED;  // (the ratio of two separate cubes)
        const SamplerF32<int> s{static_cast<const float *>(v.data), v.nx, v.ny, v.nz, v.nx, v.nx * v.ny};
        return slab_launch<ElemF32>(mode, s, v.data, cam, a, st);
    }
    case SHW_F32_PAIR: {
        if (!ratio || v.nx % 2 != 0) return SHW_EUNSUPPORTED;
        const SamplerF32Pair<int> s{static_cast<const float2 *>(v.data), v.nx, v.ny, v.nz, v.nx, v.nx * v.ny};
        return slab_launch<ElemF32Pair>(mode, s, v.data, cam, a, st);
    }
    case SHW_BF16:
    case SHW_F16:
        if (ratio || v.nx % 8 != 0) return SHW_EUNSUPPORTED;
        return render_slab_h16(mode, v, cam, a, st);
    case SHW_BF16_PAIR:
    case SHW_F16_PAIR:
        if (!ratio || v.nx % 4 != 0) return SHW_EUNSUPPORTED;
        return render_slab_h16(mode, v, cam, a, st);
    default: return SHW_EUNSUPPORTED;
    }
}

}  // namespace shw
