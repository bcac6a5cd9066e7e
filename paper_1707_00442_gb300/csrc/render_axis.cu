// render_axis.cu -- host side of the plane sweep for orthographic views down the
// spectral axis (the moment-map view of Section 2.2): eligibility, the pixel -> (x, y)
// map of the parallel projection (Appendix A), the staged box, and the launch.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "render_axis.cuh"

namespace shw {

// The sweep applies to a float32 cube seen orthographically down +-z with the image
// plane spanned by x and y, for single-cube modes.
static bool axis_eligible(const shw_volume &v, const shw_camera &c, int mode)
{
    if (debug(SHW_DEBUG_NO_AXIS_SWEEP)) return false;
    return v.storage == SHW_F32 && mode != SHW_RATIO && mode <= SHW_MOMENT1 && c.ortho && c.fwd[0] == 0.0f && c.fwd[1] == 0.0f &&
           c.fwd[2] != 0.0f && c.right[2] == 0.0f && c.up[2] == 0.0f && v.nx % 4 == 0 && aligned(v.data, 16) &&
           (long long)v.nx * v.ny < (1ll << 29);  // byte offsets in a plane fit an int
}

shw_status render_axis(int mode, int interp, const shw_volume &v, const shw_camera &c, const RenderArgs &a,
                       cudaStream_t st)
{
    if (!axis_eligible(v, c, mode)) return SHW_EUNSUPPORTED;
    // (a per-sample filter would sit in the sweep's innermost loop: filtered views take the
    // general marcher)
    if (a.filter != SHW_FILTER_NONE || a.smooth != SHW_SMOOTH_NONE) return SHW_EUNSUPPORTED;
    // pixel -> (x, y) is affine for a parallel projection
    const double W = c.width, H = c.height, aspect = W / H;
    const double hw = (double)c.ortho_half_h * aspect, hh = c.ortho_half_h;
    const double ax = 2.0 * hw * c.right[0] / W, bx = -2.0 * hh * c.up[0] / H;
    const double ay = 2.0 * hw * c.right[1] / W, by = -2.0 * hh * c.up[1] / H;
    const double cx = c.eye[0] + hw * c.right[0] * (1.0 - W) / W + hh * c.up[0] * (H - 1.0) / H;
    const double cy = c.eye[1] + hw * c.right[1] * (1.0 - W) / W + hh * c.up[1] * (H - 1.0) / H;
    const double ext_x = (kAxTX - 1) * std::fabs(ax) + (kAxTY - 1) * std::fabs(bx);
    const double ext_y = (kAxTX - 1) * std::fabs(ay) + (kAxTY - 1) * std::fabs(by);
    AxisArgs A{};
    // the tile's footprint plus margins: 2 voxels each side for FP32 rounding of the box
    // corner and the interpolation neighbour, and up to 3 to align the x start to 16 bytes
    A.bw = ((int)std::ceil(ext_x) + 8 + 3) & ~3;
    A.bh = (int)std::ceil(ext_y) + 6;
    const bool fix = A.bw <= kFixBW && A.bh <= kFixBH;
    if (fix) {
        A.bw = kFixBW;
        A.bh = kFixBH;
    }
    if (A.bw > 256 || A.bh > 256) return SHW_EUNSUPPORTED;  // the tensor copy's box limit
    A.stage_stride = fix ? kFixStride : (A.bw * A.bh + 31) & ~31;  // TMA destinations start on 128 bytes
    const int kmode = (mode == SHW_MIP && a.index == nullptr) ? kMipValue : mode;
    const size_t smem = (size_t)axis_stages(kmode, fix) * A.stage_stride * 4;
    if (smem > (size_t)kAxSmemLimit) return SHW_EUNSUPPORTED;
    A.nx = v.nx;
    A.ny = v.ny;
    A.nz = v.nz;
    A.cx = (float)cx;
    A.ax = (float)ax;
    A.bx = (float)bx;
    A.cy = (float)cy;
    A.ay = (float)ay;
    A.by = (float)by;
    A.err = device_error_word();
    A.tiles_x = ceil_div(c.width, kAxTX);
    const long long tiles = (long long)A.tiles_x * ceil_div(c.height, kAxTY);
    const float *data = static_cast<const float *>(v.data);
    CUtensorMap map;
    if (!encode_tmap_3d_f32(&map, data, v.nx, v.ny, v.nz, A.bw, A.bh)) return SHW_EUNSUPPORTED;
    const bool up = c.fwd[2] > 0.0f;  // rays advance towards +z (the sign of every ray's z step)
    return fix ? launch_axis<true>(kmode, interp, up, map, data, c, a, A, (unsigned)tiles, smem, st)
               : launch_axis<false>(kmode, interp, up, map, data, c, a, A, (unsigned)tiles, smem, st);
}

}  // namespace shw
