// render_smooth_lat.cu -- marcher instances for the in-ray box on the sample lattice (a step
// of 1/2 voxel, single-cube modes; Algorithm 8 as running sums), float32 cubes.
#include "render_impl.cuh"

namespace shw {

shw_status render_smooth_lat_f32(int mode, int interp, const shw_volume &v, const shw_camera &cam,
                                 const RenderArgs &a, cudaStream_t st)
{
    const long long nvox = (long long)v.nx * v.ny * v.nz;
    if (nvox < (1LL << 31)) {
        SamplerF32<int> s{static_cast<const float *>(v.data), v.nx, v.ny, v.nz, v.nx, v.nx * v.ny};
        return launch_render_modes<2>(mode, interp, s, s, cam, a, st);
    }
    SamplerF32<long long> s{static_cast<const float *>(v.data), v.nx, v.ny, v.nz, (long long)v.nx,
                            (long long)v.nx * v.ny};
    return launch_render_modes<2>(mode, interp, s, s, cam, a, st);
}

}  // namespace shw
