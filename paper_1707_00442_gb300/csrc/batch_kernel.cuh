// batch_kernel.cuh -- the persistent kernels of batch plans: CTAs pop (item, image tile)
// work items from an atomic counter and render each tile with the per-ray code of
// shw_render.  One kernel reads one kind of item: K = 0 float32 cubes, K = 32 or 16
// bfloat16 / binary16 bricks of that edge (32: shw_pack_bricks; 16: only bricks that a
// plan packed itself).  A kernel that read both float32 cubes and bricks would hold the
// registers of both paths (191-194 against 124-128 for either alone, trilinear), so a
// batch with both runs one kernel per kind, one after the other, each over its own work
// list.  Instances: batch.cu (K = 0), batch_b32.cu and batch_b16.cu, compiled in parallel.
#pragma once

#include "render_impl.cuh"

namespace shw {

struct BatchItemDev {
    const void *data;
    float4 *rgba;
    int nx, ny, nz, storage, mode, tiles_x, nbx, nby, nmax, brick;  // brick: edge of a brick item
    shw_camera cam;
};

struct BatchShared {
    const float4 *lut;
    float step, lo, inv_range, opacity_scale, term_alpha;
    int nwork;
};

template <int INTERP, class S>
__device__ __forceinline__ void batch_pixel(const S &s, const BatchItemDev &it, const RenderArgs &a,
                                            const float4 *lut_s, int px, int py)
{
    switch (it.mode) {
    case SHW_MIP: render_pixel<SHW_MIP, INTERP, S>(s, s, it.cam, a, lut_s, px, py); break;
    case SHW_AVG: render_pixel<SHW_AVG, INTERP, S>(s, s, it.cam, a, lut_s, px, py); break;
    case SHW_COMPOSITE: render_pixel<SHW_COMPOSITE, INTERP, S>(s, s, it.cam, a, lut_s, px, py); break;
    default: render_pixel<SHW_SPECTRAL, INTERP, S>(s, s, it.cam, a, lut_s, px, py); break;
    }
}

template <int TILE, int INTERP, int K>
__global__ void __launch_bounds__(TILE *TILE) batch_kernel(const BatchItemDev *__restrict__ items,
                                                           const int2 *__restrict__ work, int *counter, BatchShared sh)
{
    static_assert(K == 0 || K == 16 || K == 32, "float32 items, or bricks of edge 16 or 32");
    __shared__ float4 lut_s[kLut];
    __shared__ int w_s;
    for (int i = threadIdx.x; i < kLut; i += blockDim.x) lut_s[i] = sh.lut[i];
    constexpr int WX = TILE / 8;  // warps across a tile row; each warp covers 8 x 4 pixels
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = (warp % WX) * 8 + (lane & 7), ly = (warp / WX) * 4 + (lane >> 3);
    for (;;) {
        __syncthreads();  // everyone has read w_s (and the colour map is loaded)
        if (threadIdx.x == 0) w_s = atomicAdd(counter, 1);
        __syncthreads();
        const int w = w_s;
        if (w >= sh.nwork) break;
        const int2 wi = work[w];
        const BatchItemDev it = items[wi.x];
        const int px = (wi.y % it.tiles_x) * TILE + lx, py = (wi.y / it.tiles_x) * TILE + ly;
        if (px >= it.cam.width || py >= it.cam.height) continue;
        RenderArgs a{};
        a.rgba = it.rgba;
        a.lut = sh.lut;
        a.width = it.cam.width;
        a.height = it.cam.height;
        a.ckpt_interval = 64;
        a.nmax = it.nmax;
        a.step = sh.step;
        a.lo = sh.lo;
        a.inv_range = sh.inv_range;
        a.opacity_scale = sh.opacity_scale;
        a.term_alpha = sh.term_alpha;
        a.nx = it.nx;
        a.ny = it.ny;
        a.nz = it.nz;
        if constexpr (K == 0) {
            const SamplerF32<int> s{static_cast<const float *>(it.data), it.nx, it.ny, it.nz, it.nx, it.nx * it.ny};
            batch_pixel<INTERP>(s, it, a, lut_s, px, py);
        } else {
            // 32-bit element offsets: the plans admit brick items of fewer than 2^31 elements
            if (it.storage == SHW_BF16_BRICK) {
                const SamplerBrick<__nv_bfloat16, int, K> s{static_cast<const unsigned short *>(it.data), it.nx, it.ny,
                                                            it.nz, it.nbx, it.nby};
                batch_pixel<INTERP>(s, it, a, lut_s, px, py);
            } else {
                const SamplerBrick<__half, int, K> s{static_cast<const unsigned short *>(it.data), it.nx, it.ny, it.nz,
                                                     it.nbx, it.nby};
                batch_pixel<INTERP>(s, it, a, lut_s, px, py);
            }
        }
    }
}

using BatchKernel = void (*)(const BatchItemDev *, const int2 *, int *, BatchShared);

// The kernel for a tile edge (8 or 16), an interpolation and a kind of item (0: float32
// cubes; 16, 32: bfloat16 or binary16 bricks of that edge).  Every item of its work list
// must be of that kind.
BatchKernel batch_kernel_for(int tile, int interp, int kind);
BatchKernel batch_kernel_b16(int tile, int interp);  // batch_b16.cu
BatchKernel batch_kernel_b32(int tile, int interp);  // batch_b32.cu

}  // namespace shw
